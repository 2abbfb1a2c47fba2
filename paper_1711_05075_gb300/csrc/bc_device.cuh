// Device helpers shared by the kernel translation units (bc_kernels.cu,
// bc_binned.cu).  Not part of the public interface.
#pragma once
#include <climits>
#include <utility>
#include <cuda_runtime.h>

#include "bc_fft.cuh"
#include "bc_internal.h"

namespace bc {

constexpr int TB = 256; // threads per transform block
constexpr int CL = 16;  // interleaved lines per tile (16 complex = 128 bytes per tile row)

// Block loop over the work items of a sequence of instances (or pairs),
// giving each block of the grid an even share across them.
struct RotStart {
    int rot = 0;
    __device__ __forceinline__ int first() const
    {
        const int st = rot % (int)gridDim.x;
        return ((int)blockIdx.x - st + (int)gridDim.x) % (int)gridDim.x;
    }
};

template <int NF>
__device__ __forceinline__ void load_twiddles(float2 *dst, const float2 *__restrict__ src)
{
    for (int k = threadIdx.x; k < NF; k += blockDim.x) dst[k] = src[k];
}

// Kaiser-Bessel window phi(v) = I0(beta sqrt(1 - s^2)) / I0(beta), s = 2v/W,
// on |s| <= 1 (fine-grid cells), as piecewise polynomials.  A knot at u has stencil cells
// g0 + t, t < W, g0 = ceil(u - W/2); with x = u - g0 - (W/2 - 1) in (0, 1] the
// weight of cell g0 + t is phi(x + W/2 - 1 - t), a smooth function of x on
// [0, 1] for each t (phi is a power series in 1 - s^2 inside its support).
// Each piece is replaced by its degree-KB_DEG interpolant at Chebyshev nodes,
// written in powers of y = x - 1/2 and evaluated by Horner's rule in FP32
// (piecewise-polynomial kernel evaluation as in Barnett, Magland and af
// Klinteberg, SIAM J. Sci. Comput. 2019).  The coefficients are built in FP64
// from the closed form (k_build_tables); for W = 6, 8, 10 at their default
// beta the FP32 evaluation stays within 1e-7 of phi (phi <= 1).
__device__ __forceinline__ float kb_poly(const float (&c)[KB_NC], float x)
{
    const float y = x - 0.5f;
    float acc = c[KB_DEG];
#pragma unroll
    for (int m = KB_DEG - 1; m >= 0; m--) acc = fmaf(acc, y, c[m]);
    return acc;
}

// Coefficients of piece t (consts + KB_OFF + t KB_NC) into registers.
__device__ __forceinline__ void kb_load(const float *__restrict__ consts, int t, float (&c)[KB_NC])
{
#pragma unroll
    for (int m = 0; m < KB_NC; m++) c[m] = consts[KB_OFF + t * KB_NC + m];
}

// Transform of the indicator of a ball of radius r at angular wavenumber k
// (Sec. 2.5): 4 pi (sin kr - kr cos kr) / k^3, and for x = kr < 0.5 the
// Maclaurin series 4 pi r^3 (1/3 - x^2/30 + x^4/840 - x^6/45360 + x^8/3991680)
// (the next term is below 2e-12 relative).  FP64.
__device__ __forceinline__ double ball_ft64(double r, double k)
{
    const double pi = 3.14159265358979323846;
    const double x = k * r;
    if (x < 0.5) {
        const double x2 = x * x;
        return 4.0 * pi * r * r * r *
               (1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0 - x2 * x2 * x2 / 45360.0 + x2 * x2 * x2 * x2 / 3991680.0);
    }
    return 4.0 * pi * (sin(x) - x * cos(x)) / (k * k * k);
}

// Support box of instance i -> its plan (the box accumulators are reset for
// the next launch).  A box larger than the instance's capacity raises the
// error word and the instance is treated as empty.
__device__ __forceinline__ void plan_instance(const Geometry &g, const InstDesc *__restrict__ inst, int i, int *bb,
                                              InstPlan *plan, int *err)
{
    int L0[3], H0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        L0[a] = __ldcg(&bb[8 * i + a]); // written by other blocks' atomics: read at L2
        H0[a] = __ldcg(&bb[8 * i + 3 + a]);
        bb[8 * i + a] = INT_MAX;
        bb[8 * i + 3 + a] = INT_MIN;
    }
    InstPlan pl;
    bool empty = inst[i].nknots <= 0 || L0[0] == INT_MAX;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int b = empty ? 0 : min(H0[a] - L0[a] + 1, g.n);
        if (b > inst[i].cap_e) {
            atomicOr(err, 1);
            empty = true;
        }
        pl.lo[a] = empty ? 0 : L0[a];
        pl.b[a] = b;
        pl.pos0[a] = empty ? 0 : ((L0[a] % g.n) + g.n) % g.n;
    }
    if (empty) pl.b[0] = pl.b[1] = pl.b[2] = 0;
    pl.bzp = (pl.b[2] + 3) & ~3;
    plan[i] = pl;
}

// Blocks per launch: the number that can be resident on the device at once.
template <typename K>
static int resident_blocks(K kernel, size_t smem, int nsm, int threads = TB)
{
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
    return per * nsm;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

// Programmatic dependent launch.  A pass launched as a programmatic dependent
// of the kernel before it on the stream may start once every block of that
// kernel has signalled (pdl_signal) or exited: its blocks become resident as
// the earlier kernel's blocks leave their SMs and run the prologue that reads
// only the context's constant tables.  pdl_wait then holds every thread until
// the earlier kernel has completed and its writes are visible; everything a
// pass reads from earlier passes is read after it.  Both are no-ops for a
// kernel launched the ordinary way.  The earlier kernel's signal cannot starve
// it: the dependent launch needs all of its blocks to have started.
__device__ __forceinline__ void pdl_signal() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// kernel<<<grid, threads, smem, s>>>(args...), as a programmatic dependent of
// the previous kernel on s when `dependent` is set.
template <typename... P, typename... A>
static cudaError_t launch_k(void (*kernel)(P...), int grid, int threads, size_t smem, cudaStream_t s, bool dependent,
                            A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

} // namespace bc
