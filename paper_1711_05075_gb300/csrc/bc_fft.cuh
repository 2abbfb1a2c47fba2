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
#include <cuda_bf16.h>
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

// x * exp(-+2 pi i E / 16) for the exponents a radix-16 butterfly uses
// (E = n2 k1, n2, k1 < 4).  E = 0 and 4 are exact (identity, -+i); E = 2 and 6
// take two adds and two multiplies by sqrt(1/2); the rest a complex multiply.
template <int E, bool INV>
__device__ __forceinline__ float2 tw16_mul(float2 x)
{
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    const float sg = INV ? -1.f : 1.f; // imaginary part of the twiddle flips for the inverse
    if constexpr (E == 0) {
        return x;
    } else if constexpr (E == 4) {
        return mul_mi<INV>(x);
    } else if constexpr (E == 2) { // (1 -+ i) h
        return INV ? make_float2(h * (x.x - x.y), h * (x.x + x.y)) : make_float2(h * (x.x + x.y), h * (x.y - x.x));
    } else if constexpr (E == 6) { // (-1 -+ i) h
        return INV ? make_float2(-h * (x.x + x.y), h * (x.x - x.y)) : make_float2(h * (x.y - x.x), -h * (x.x + x.y));
    } else if constexpr (E == 1) {
        return cmul(x, make_float2(c1, -sg * s1));
    } else if constexpr (E == 3) {
        return cmul(x, make_float2(s1, -sg * c1));
    } else {
        static_assert(E == 9, "radix-16 twiddle exponent");
        return cmul(x, make_float2(-c1, sg * s1));
    }
}

template <int N2, int K1, bool INV>
__device__ __forceinline__ float2 tw16_apply(float2 x) { return tw16_mul<N2 * K1, INV>(x); }

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
            for (int k1 = 0; k1 < 4; k1++) y[n2][k1] = t[k1];
        }
        y[1][1] = tw16_apply<1, 1, INV>(y[1][1]);
        y[1][2] = tw16_apply<1, 2, INV>(y[1][2]);
        y[1][3] = tw16_apply<1, 3, INV>(y[1][3]);
        y[2][1] = tw16_apply<2, 1, INV>(y[2][1]);
        y[2][2] = tw16_apply<2, 2, INV>(y[2][2]);
        y[2][3] = tw16_apply<2, 3, INV>(y[2][3]);
        y[3][1] = tw16_apply<3, 1, INV>(y[3][1]);
        y[3][2] = tw16_apply<3, 2, INV>(y[3][2]);
        y[3][3] = tw16_apply<3, 3, INV>(y[3][3]);
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

// Radix schedules: S = 0 the default of each size, S = 1 an alternative for
// the forward passes (chosen by measurement; every last stage has a radix
// divisible by 4, which the pruned x pass needs).
template <int NF, int S = 0>
struct Radix;
template <> struct Radix<32, 0>  { static constexpr int r0 = 4, r1 = 8, r2 = 1; };
template <> struct Radix<64, 0>  { static constexpr int r0 = 8, r1 = 8, r2 = 1; };
template <> struct Radix<96, 0>  { static constexpr int r0 = 3, r1 = 4, r2 = 8; };
template <> struct Radix<128, 0> { static constexpr int r0 = 8, r1 = 16, r2 = 1; };
template <> struct Radix<192, 0> { static constexpr int r0 = 3, r1 = 8, r2 = 8; };
template <> struct Radix<256, 0> { static constexpr int r0 = 16, r1 = 16, r2 = 1; };
template <> struct Radix<512, 0> { static constexpr int r0 = 8, r1 = 8, r2 = 8; };
template <> struct Radix<64, 1>  { static constexpr int r0 = 4, r1 = 16, r2 = 1; };
template <> struct Radix<128, 1> { static constexpr int r0 = 16, r1 = 8, r2 = 1; };
template <> struct Radix<192, 1> { static constexpr int r0 = 3, r1 = 4, r2 = 16; };
template <> struct Radix<256, 1> { static constexpr int r0 = 4, r1 = 8, r2 = 8; };
template <> struct Radix<512, 1> { static constexpr int r0 = 8, r1 = 4, r2 = 16; };

// Schedule of the split-precision passes: the default of each length, except
// 256, whose default (16.16) has no radix-8 stage for the tensor cores.
template <int NF>
struct SplitSched {
    static constexpr int S = NF == 256 ? 1 : 0;
};

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
    // Writes the loaded values to their positions of a tile (tile[pos * C + c]).
    __device__ __forceinline__ void scatter(float2 *tile) const
    {
#pragma unroll
        for (int it = 0; it < IT; it++) {
            const int idx = (int)threadIdx.x + it * NT;
            if ((TOT % NT) != 0 && idx >= TOT) break;
            const int c = idx % C, j = idx / C;
#pragma unroll
            for (int r = 0; r < R; r++) tile[(j + r * NB) * C + c] = v[it][r];
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
template <int NF, int S = 0>
struct LastStage {
    static constexpr int R = Radix<NF, S>::r2 > 1 ? Radix<NF, S>::r2 : Radix<NF, S>::r1;
    static constexpr int NS = NF / R;
};

// The middle (three-stage schedules) and last stages after rr_first has
// written tile s0; s1 is scratch for three-stage schedules.  All threads call
// it; the caller adds a barrier before s0/s1 are written again.
template <int NF, bool INV, int C, int NT, int S = 0, class Sink>
__device__ __forceinline__ void rr_rest(float2 *s0, float2 *s1, const float2 *tw, Sink sink)
{
    using R = Radix<NF, S>;
    if constexpr (R::r2 > 1) {
        il_stage<NF, R::r1, R::r0, INV, C, NT>(s0, s1, tw);
        __syncthreads();
        rr_last<NF, R::r2, R::r0 * R::r1, INV, C, NT>(s1, tw, sink);
    } else {
        rr_last<NF, R::r1, R::r0, INV, C, NT>(s0, tw, sink);
    }
}

// ---------------------------------------------------------------------------
// Split-precision radix-8 stage on the tensor cores.  The 8-point DFT of a
// butterfly is y = F x with F[r'][r] = exp(-+2 pi i r r' / 8); with complex
// numbers as (re, im) pairs it is a 16 x 16 real matrix acting on a 16-vector,
// so one mma.m16n8k16 (A = F, B = the inputs of 8 butterflies, one per column)
// transforms 8 butterflies.  Both F and the twiddled inputs are split into
// BF16 hi + lo parts (hi = bf16(v), lo = bf16(v - hi)); the product is formed
// as F_hi x_hi + F_hi x_lo + F_lo x_hi with FP32 accumulation (the lo x lo term,
// of relative size 2^-32, is dropped).  Lane (g, t) of a warp loads inputs
// r = t and r = t + 4 of butterfly g of the group (the B fragment layout) and
// receives output components g and g + 8 of butterflies 2t and 2t + 1.
__device__ __forceinline__ float dft8_entry(int m, int k, bool inv)
{
    // A[m][k], m = 2 r' + p, k = 2 r + q: the 2 x 2 real block of exp(-+i theta), theta = 2 pi r r' / 8
    const float h = 0.70710678118654752440f;
    const int e = ((m >> 1) * (k >> 1)) & 7;
    // cos and sin of e pi / 4
    const float c = e == 0 ? 1.f : e == 4 ? -1.f : (e == 2 || e == 6) ? 0.f : (e == 1 || e == 7) ? h : -h;
    const float sv = e == 2 ? 1.f : e == 6 ? -1.f : (e == 0 || e == 4) ? 0.f : (e == 1 || e == 3) ? h : -h;
    const float s = inv ? -sv : sv;
    const int p = m & 1, q = k & 1;
    return p == 0 ? (q == 0 ? c : s) : (q == 0 ? -s : c);
}

__device__ __forceinline__ unsigned bf2(float lo_elem, float hi_elem)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem); // .x = first (lower 16 bits)
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ void split_bf16(float v, float &hi, float &lo)
{
    hi = __bfloat162float(__float2bfloat16_rn(v));
    lo = v - hi;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int NF, int NS, bool INV, int C, int NT>
__device__ __forceinline__ void tc_stage8(const float2 *__restrict__ in, float2 *__restrict__ out,
                                          const float2 *__restrict__ tw)
{
    constexpr int R = 8, NB = NF / R, TOT = NB * C, GROUPS = TOT / 8;
    static_assert(TOT % 8 == 0, "groups of 8 butterflies");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // A fragments of F, split into hi and lo
    unsigned ahi[4], alo[4];
    {
        const int mm[4] = {g, g + 8, g, g + 8};
        const int kk[4] = {2 * t, 2 * t, 2 * t + 8, 2 * t + 8};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float h0, l0, h1, l1;
            split_bf16(dft8_entry(mm[i], kk[i], INV), h0, l0);
            split_bf16(dft8_entry(mm[i], kk[i] + 1, INV), h1, l1);
            ahi[i] = bf2(h0, h1);
            alo[i] = bf2(l0, l1);
        }
    }
    float *outf = reinterpret_cast<float *>(out);
    for (int grp = warp; grp < GROUPS; grp += NT / 32) {
        // inputs r = t and r = t + 4 of butterfly b = 8 grp + g
        const int b = grp * 8 + g;
        const int c = b % C, j = b / C, k = j % NS;
        float2 x0 = in[(j + t * NB) * C + c];
        float2 x1 = in[(j + (t + 4) * NB) * C + c];
        if (NS > 1) {
            if (t > 0) {
                float2 w = tw[t * k * (NF / (NS * R))];
                if (INV) w.y = -w.y;
                x0 = cmul(x0, w);
            }
            float2 w = tw[(t + 4) * k * (NF / (NS * R))];
            if (INV) w.y = -w.y;
            x1 = cmul(x1, w);
        }
        float h0, l0, h1, l1, h2, l2, h3, l3;
        split_bf16(x0.x, h0, l0);
        split_bf16(x0.y, h1, l1);
        split_bf16(x1.x, h2, l2);
        split_bf16(x1.y, h3, l3);
        const unsigned bh0 = bf2(h0, h1), bh1 = bf2(h2, h3), bl0 = bf2(l0, l1), bl1 = bf2(l2, l3);
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(d, ahi, bh0, bh1);
        mma_bf16(d, ahi, bl0, bl1);
        mma_bf16(d, alo, bh0, bh1);
        // d[0] = C[g][2t], d[1] = C[g][2t+1], d[2] = C[g+8][2t], d[3] = C[g+8][2t+1]
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int bb = grp * 8 + 2 * t + u;
            const int cc = bb % C, jj = bb / C, kk2 = jj % NS;
            const int base = (jj / NS) * NS * R + kk2;
            const int p = g & 1, r0 = g >> 1;
            outf[((base + r0 * NS) * C + cc) * 2 + p] = d[u];
            outf[((base + (r0 + 4) * NS) * C + cc) * 2 + p] = d[2 + u];
        }
    }
}

// A stage of the split-precision schedule: tensor-core DFT for radix 8, FP32 otherwise.
template <int NF, int R, int NS, bool INV, int C, int NT>
__device__ __forceinline__ void sp_stage(const float2 *in, float2 *out, const float2 *tw)
{
    if constexpr (R == 8) tc_stage8<NF, NS, INV, C, NT>(in, out, tw);
    else il_stage<NF, R, NS, INV, C, NT>(in, out, tw);
}

// Split-precision transform of a tile whose inputs were scattered into s0 by
// FirstInputs::scatter (natural order, whatever the loading schedule); then
// sink(it, r, c, pos, value) in the thread mapping of rr_last for radix
// schedule S.  All threads call it; the caller adds a barrier before s0/s1 are
// written again.
template <int NF, bool INV, int C, int NT, int S, class Sink>
__device__ __forceinline__ void sp_all(float2 *s0, float2 *s1, const float2 *tw, Sink sink)
{
    using R = Radix<NF, S>;
    sp_stage<NF, R::r0, 1, INV, C, NT>(s0, s1, tw);
    __syncthreads();
    sp_stage<NF, R::r1, R::r0, INV, C, NT>(s1, s0, tw);
    __syncthreads();
    const float2 *fin = s0;
    if constexpr (R::r2 > 1) {
        sp_stage<NF, R::r2, R::r0 * R::r1, INV, C, NT>(s0, s1, tw);
        __syncthreads();
        fin = s1;
    }
    constexpr int RL = LastStage<NF, S>::R, NSL = LastStage<NF, S>::NS, TOT = NSL * C, IT = (TOT + NT - 1) / NT;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int idx = (int)threadIdx.x + it * NT;
        if ((TOT % NT) != 0 && idx >= TOT) break;
        const int c = idx % C, j = idx / C;
#pragma unroll
        for (int r = 0; r < RL; r++) sink(it, r, c, j + r * NSL, fin[(j + r * NSL) * C + c]);
    }
}

} // namespace bc
