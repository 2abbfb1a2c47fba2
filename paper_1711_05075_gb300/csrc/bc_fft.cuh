// Batched one-dimensional FFTs in shared memory (FP32), used by every
// transform pass of the correlation.
//
// Algorithm: the self-sorting Stockham formulation of the Cooley-Tukey FFT
// (T. G. Stockham, 1966; as arranged for GPUs by Govindaraju et al.,
// "High performance discrete Fourier transforms on graphics processors",
// SC 2008).  A length-NF transform runs as a sequence of radix-R stages; with
// Ns the product of the radices already applied, butterfly j of a stage reads
// x[j + r NF/R] (r < R), multiplies input r by w^(r (j mod Ns) NF/(Ns R)),
// applies an R-point DFT and writes y[(j div Ns) Ns R + (j mod Ns) + r Ns].
// Output is in natural order after the last stage; stages ping-pong between
// two shared-memory tiles.  Radix schedules: 32 = 4.8, 64 = 8.8,
// 96 = 3.4.8, 128 = 8.16, 192 = 3.8.8, 256 = 16.16, 512 = 8.8.8.
//
// Direction: forward uses exp(-2 pi i jk/NF), inverse exp(+2 pi i jk/NF); no
// scaling.  The twiddle table holds exp(-2 pi i k/NF), k < NF, rounded once
// from FP64; the inverse conjugates it.
#pragma once
#include <cuda_runtime.h>

namespace bc {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// exp(-+2 pi i e / 16) for the exponents a radix-16 butterfly uses (e = 0..9)
template <bool INV>
__device__ __forceinline__ float2 tw16(int e)
{
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    float2 w;
    switch (e) {
    case 0: w = make_float2(1.f, 0.f); break;
    case 1: w = make_float2(c1, -s1); break;
    case 2: w = make_float2(h, -h); break;
    case 3: w = make_float2(s1, -c1); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 6: w = make_float2(-h, -h); break;
    case 9: w = make_float2(-c1, s1); break;
    default: w = make_float2(1.f, 0.f); break; // not used
    }
    if (INV) w.y = -w.y;
    return w;
}

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2 *v)
{
    if constexpr (R == 2) {
        float2 t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    } else if constexpr (R == 3) {
        // exp(-+2 pi i/3) = -1/2 -+ i sqrt(3)/2
        const float s = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
        float2 t1 = cadd(v[1], v[2]);
        float2 t2 = csub(v[1], v[2]);
        float2 m = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
        float2 r = make_float2(-s * t2.y, s * t2.x); // i s t2
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    } else if constexpr (R == 4) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, b1);
        v[3] = csub(a1, b1);
    } else if constexpr (R == 16) {
        // 16 = 4 x 4: index n = 4 n1 + n2, k = k1 + 4 k2; 4-point DFTs over n1,
        // twiddles exp(-+2 pi i n2 k1 / 16), then 4-point DFTs over n2.
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) {
            float2 t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
            dft_small<4, INV>(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; k1++) y[n2][k1] = cmul(t[k1], tw16<INV>(n2 * k1));
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) {
            float2 t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            dft_small<4, INV>(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = t[k2];
        }
    } else if constexpr (R == 8) {
        const float h = 0.70710678118654752440f;
        float2 a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            a[k] = cadd(v[k], v[k + 4]);
            b[k] = csub(v[k], v[k + 4]);
        }
        // b[k] *= exp(-+2 pi i k / 8)
        b[1] = INV ? make_float2(h * (b[1].x - b[1].y), h * (b[1].x + b[1].y))
                   : make_float2(h * (b[1].x + b[1].y), h * (b[1].y - b[1].x));
        b[2] = mul_mi<INV>(b[2]);
        b[3] = INV ? make_float2(-h * (b[3].x + b[3].y), h * (b[3].x - b[3].y))
                   : make_float2(h * (b[3].y - b[3].x), -h * (b[3].x + b[3].y));
        dft_small<4, INV>(a);
        dft_small<4, INV>(b);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[2 * k] = a[k];
            v[2 * k + 1] = b[k];
        }
    }
}

template <int NF>
struct Radix;
template <> struct Radix<32>  { static constexpr int r0 = 4, r1 = 8, r2 = 1; };
template <> struct Radix<64>  { static constexpr int r0 = 8, r1 = 8, r2 = 1; };
template <> struct Radix<96>  { static constexpr int r0 = 3, r1 = 4, r2 = 8; };
template <> struct Radix<128> { static constexpr int r0 = 8, r1 = 16, r2 = 1; };
template <> struct Radix<192> { static constexpr int r0 = 3, r1 = 8, r2 = 8; };
template <> struct Radix<256> { static constexpr int r0 = 16, r1 = 16, r2 = 1; };
template <> struct Radix<512> { static constexpr int r0 = 8, r1 = 8, r2 = 8; };

// ---------------------------------------------------------------------------
// Interleaved tiles: C lines stored as x[pos * C + c].  Consecutive threads take
// consecutive lines c of the same butterfly, so every shared-memory access of
// a stage is a run of C consecutive complex values (no bank conflicts), and a
// tile row of C values is one 8C-byte run in global memory as well.
template <int NF, int R, int NS, bool INV, int C, int NT>
__device__ __forceinline__ void il_stage(const float2 *__restrict__ in, float2 *__restrict__ out,
                                         const float2 *__restrict__ tw)
{
    constexpr int NB = NF / R;
    constexpr int TOT = NB * C;
    constexpr int IT = (TOT + NT - 1) / NT;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = (int)threadIdx.x + it * NT;
        if ((TOT % NT) != 0 && idx >= TOT) break;
        const int c = idx % C, j = idx / C;
        const int k = j % NS;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            float2 x = in[(j + r * NB) * C + c];
            if (NS > 1 && r > 0) {
                float2 w = tw[r * k * (NF / (NS * R))];
                if (INV) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        dft_small<R, INV>(v);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) out[(base + r * NS) * C + c] = v[r];
    }
}

// Transforms the C interleaved lines of tile `a` (b: scratch tile); all NT
// threads of the block must call it.  Returns the tile holding the result;
// ends with a block barrier.
template <int NF, bool INV, int C, int NT>
__device__ __forceinline__ float2 *il_fft(float2 *a, float2 *b, const float2 *tw)
{
    using RR = Radix<NF>;
    il_stage<NF, RR::r0, 1, INV, C, NT>(a, b, tw);
    __syncthreads();
    il_stage<NF, RR::r1, RR::r0, INV, C, NT>(b, a, tw);
    __syncthreads();
    if constexpr (RR::r2 > 1) {
        il_stage<NF, RR::r2, RR::r0 * RR::r1, INV, C, NT>(a, b, tw);
        __syncthreads();
        return b;
    } else {
        return a;
    }
}

// ---------------------------------------------------------------------------
// Register-resident first and last stages.  A transform of C interleaved lines
// runs as: first stage (inputs held in registers, loaded straight from global
// memory by the caller) -> shared tile -> middle stage (only for three-stage
// schedules, shared -> shared) -> last stage (shared -> registers -> a sink
// functor).  Shared memory then carries each value once per exchange instead
// of once per stage plus a gather and a scatter.

// Inputs of the first stage owned by the calling thread: butterfly (c, j) of
// iteration `it` needs positions j + r NF/R, r < R.
template <int NF, int R, int C, int NT>
struct FirstInputs {
    static constexpr int NB = NF / R, TOT = NB * C, IT = (TOT + NT - 1) / NT;
    float2 v[IT][R];
    // src(c, pos) -> float2: value of line c at position pos (issue the loads only).
    template <class Src>
    __device__ __forceinline__ void load(Src src)
    {
#pragma unroll
        for (int it = 0; it < IT; it++) {
            const int idx = (int)threadIdx.x + it * NT;
            const int c = idx % C, j = idx / C;
#pragma unroll
            for (int r = 0; r < R; r++)
                v[it][r] = ((TOT % NT) == 0 || idx < TOT) ? src(c, j + r * NB) : make_float2(0.f, 0.f);
        }
    }
    // visit(c, pos) for every position load() read.
    template <class Vis>
    __device__ __forceinline__ void for_each(Vis visit) const
    {
#pragma unroll
        for (int it = 0; it < IT; it++) {
            const int idx = (int)threadIdx.x + it * NT;
            if ((TOT % NT) != 0 && idx >= TOT) break;
            const int c = idx % C, j = idx / C;
#pragma unroll
            for (int r = 0; r < R; r++) visit(c, j + r * NB);
        }
    }
};

// First stage (Ns = 1, no twiddles): registers -> out[pos * C + c].
template <int NF, int R, bool INV, int C, int NT>
__device__ __forceinline__ void rr_first(const FirstInputs<NF, R, C, NT> &in, float2 *__restrict__ out)
{
    using FI = FirstInputs<NF, R, C, NT>;
#pragma unroll
    for (int it = 0; it < FI::IT; it++) {
        const int idx = (int)threadIdx.x + it * NT;
        if ((FI::TOT % NT) != 0 && idx >= FI::TOT) break;
        const int c = idx % C, j = idx / C;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = in.v[it][r];
        dft_small<R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; r++) out[(j * R + r) * C + c] = v[r];
    }
}

// Last stage: in[pos * C + c] -> registers -> sink(it, r, c, pos, value), where
// the output position is pos = j + r NS for butterfly j (< NS) of iteration it.
template <int NF, int R, int NS, bool INV, int C, int NT, class Sink>
__device__ __forceinline__ void rr_last(const float2 *__restrict__ in, const float2 *__restrict__ tw, Sink sink)
{
    constexpr int NB = NF / R;
    static_assert(NB == NS, "last stage");
    constexpr int TOT = NB * C;
    constexpr int IT = (TOT + NT - 1) / NT;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = (int)threadIdx.x + it * NT;
        if ((TOT % NT) != 0 && idx >= TOT) break;
        const int c = idx % C, j = idx / C;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            float2 x = in[(j + r * NB) * C + c];
            if (r > 0) {
                float2 w = tw[r * j * (NF / (NS * R))];
                if (INV) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        dft_small<R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; r++) sink(it, r, c, j + r * NS, v[r]);
    }
}

// Radix of the last stage of a schedule and its output stride.
template <int NF>
struct LastStage {
    static constexpr int R = Radix<NF>::r2 > 1 ? Radix<NF>::r2 : Radix<NF>::r1;
    static constexpr int NS = NF / R;
};

// The middle (three-stage schedules) and last stages after rr_first has
// written tile s0; s1 is scratch for three-stage schedules.  All threads call
// it; the caller adds a barrier before s0/s1 are written again.
template <int NF, bool INV, int C, int NT, class Sink>
__device__ __forceinline__ void rr_rest(float2 *s0, float2 *s1, const float2 *tw, Sink sink)
{
    using R = Radix<NF>;
    if constexpr (R::r2 > 1) {
        il_stage<NF, R::r1, R::r0, INV, C, NT>(s0, s1, tw);
        __syncthreads();
        rr_last<NF, R::r2, R::r0 * R::r1, INV, C, NT>(s1, tw, sink);
    } else {
        rr_last<NF, R::r1, R::r0, INV, C, NT>(s0, tw, sink);
    }
}

} // namespace bc
