// bc_correlate_noalloc: the correlation of one small pair of shapes without any
// device allocation.
//
// Some callers cannot allocate device memory: plugins hosted by an
// application that owns the whole device heap and forbids cudaMalloc, and
// real-time loops that must not take the allocator's locks.  They hand in
// device buffers for the inputs and the output; everything else this entry
// point needs (tables, packed knots, support boxes, spreading boxes, transform
// planes) lives in one file-scope __device__ array of BC_NOALLOC_SCRATCH_BYTES
// (8 MiB), enough for N = 32, two radius levels and 8192 knots per shape.
// Every GPU that loads the library holds that array until the process exits.
//
// The kernels are the ones bc_correlate launches; only their scratch pointers
// differ.  All calls share the one array: two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it and give
// wrong results.  The parts that must start at a known state (the spreading
// boxes, the support-box accumulators, the status words) are reset by every call.
// Each call synchronises its stream twice -- after the knot checks, so that no
// kernel sees an out-of-range level id, and at the end, to read the kernels'
// status word -- so it cannot be recorded into a CUDA graph.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ballcorr.h"
#include "bc_internal.h"

using namespace bc;

namespace {

constexpr int kN = BC_NOALLOC_MAX_N;
constexpr int kn = 2 * kN;
constexpr int kL = BC_NOALLOC_MAX_LEVELS;
constexpr int kK = BC_NOALLOC_MAX_KNOTS;
constexpr int kH = kN / 2;
constexpr int kQ = 3 * (kN / 2) * (kN / 2) + 1;

// Byte offsets inside the scratch array (each region 256-byte aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t oRadii = 0;
constexpr size_t oDeconv = al(oRadii + sizeof(double) * kL);
constexpr size_t oBallft = al(oDeconv + sizeof(float) * kN);
constexpr size_t oTwn = al(oBallft + sizeof(float) * kL * kQ);
constexpr size_t oTwN = al(oTwn + sizeof(float2) * kn);
constexpr size_t oConsts = al(oTwN + sizeof(float2) * kN);
constexpr size_t oErr = al(oConsts + sizeof(float) * CONSTS_FLOATS);
constexpr size_t oStats = al(oErr + sizeof(int));
constexpr size_t oBoxes = al(oStats + sizeof(unsigned) * 4);
constexpr size_t oInst = al(oBoxes + sizeof(int) * 8 * 2);
constexpr size_t oPairs = al(oInst + sizeof(InstDesc) * 2);
constexpr size_t oPlan = al(oPairs + sizeof(PairDesc));
constexpr size_t oKnots = al(oPlan + sizeof(InstPlan) * 2);
constexpr size_t oKu = al(oKnots + sizeof(float4) * 2 * kK);
constexpr size_t oGrid = al(oKu + sizeof(float4) * 2 * kK);
constexpr size_t kGridBytes = sizeof(float) * 2 * kL * (size_t)kn * kn * kn;
constexpr size_t oZ1 = al(oGrid + kGridBytes);
constexpr size_t oY1 = al(oZ1 + sizeof(float2) * 2 * kL * (size_t)kn * kn * kH);
constexpr size_t oH = al(oY1 + sizeof(float2) * 2 * kL * (size_t)kn * kN * kH);
constexpr size_t kScratchBytes = al(oH + sizeof(float2) * (size_t)kN * kN * kH);
static_assert(kScratchBytes <= BC_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented size");

} // namespace

// The scratch memory: zero at module load, shared by every call in the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BC_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {}; // device address of the array, per device
int g_nsm[kMaxDevices] = {};

bc_status nfail(bc_status s, const std::string &m)
{
    set_last_error(m);
    return s;
}

bc_status ncuda(cudaError_t e, const char *where)
{
    set_last_error(std::string("bc_correlate_noalloc: ") + where + ": " + cudaGetErrorString(e));
    return BC_ERR_CUDA;
}

} // namespace

extern "C" bc_status bc_correlate_noalloc(const bc_params *p, const float *xyzA, const int *levelA, int nA,
                                          const float *xyzB, const int *levelB, int nB, const float *quat,
                                          float *out, void *cuda_stream)
{
    try {
        if (!p || !quat || !out) return nfail(BC_ERR_ARG, "bc_correlate_noalloc: null argument");
        if ((nA > 0 && (!xyzA || !levelA)) || (nB > 0 && (!xyzB || !levelB)))
            return nfail(BC_ERR_ARG, "bc_correlate_noalloc: null knot arrays");
        if (p->N != kN || p->sigma != 2 || p->precision != 0)
            return nfail(BC_ERR_ARG, "bc_correlate_noalloc: needs N = 32, sigma = 2, precision 0");
        if (p->level_count < 1 || p->level_count > kL || !p->level_radii)
            return nfail(BC_ERR_ARG, "bc_correlate_noalloc: level_count must be in [1, BC_NOALLOC_MAX_LEVELS]");
        if (nA < 0 || nB < 0 || nA > kK || nB > kK)
            return nfail(BC_ERR_ARG, "bc_correlate_noalloc: knot count outside [0, BC_NOALLOC_MAX_KNOTS]");
        if (p->W < 2 || p->W > 10 || !(p->period > 0) || !std::isfinite(p->period))
            return nfail(BC_ERR_ARG, "bc_correlate_noalloc: W must be in [2, 10] and period > 0");
        for (int l = 0; l < p->level_count; l++)
            if (!(p->level_radii[l] > 0) || !std::isfinite(p->level_radii[l]))
                return nfail(BC_ERR_ARG, "bc_correlate_noalloc: radii must be finite and > 0");
        const double qn = (double)quat[0] * quat[0] + (double)quat[1] * quat[1] + (double)quat[2] * quat[2] +
                          (double)quat[3] * quat[3];
        if (!(qn > 1e-30) || !std::isfinite(qn)) return nfail(BC_ERR_ARG, "bc_correlate_noalloc: zero quaternion");
        double beta = p->beta;
        if (!(beta > 0)) {
            const double a = (double)p->W / 2 * 1.5;
            beta = M_PI * std::sqrt(a * a - 0.8);
        }
        if (!std::isfinite(beta) || beta > 80) return nfail(BC_ERR_ARG, "bc_correlate_noalloc: beta out of range");
        beta = (double)(float)beta;

        // set-up, once per device: the device address of the scratch array
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return ncuda(e, "cudaGetDevice");
        if (dev < 0 || dev >= kMaxDevices) return nfail(BC_ERR_UNSUPPORTED, "bc_correlate_noalloc: device index");
        unsigned char *base = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_setup_mutex);
            if (!g_scratch_ptr[dev]) {
                void *ptr = nullptr;
                e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
                if (e != cudaSuccess) return ncuda(e, "cudaGetSymbolAddress");
                int nsm = 0;
                e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                if (e != cudaSuccess) return ncuda(e, "cudaDeviceGetAttribute");
                g_nsm[dev] = nsm;
                g_scratch_ptr[dev] = (unsigned char *)ptr;
            }
            base = g_scratch_ptr[dev];
        }
        const int nsm = g_nsm[dev];
        cudaStream_t st = (cudaStream_t)cuda_stream;

        Geometry g{};
        g.N = kN;
        g.n = kn;
        g.W = p->W;
        g.L = p->level_count;
        g.H = kH;
        g.prec = 0;
        g.beta = (float)beta;
        g.n_over_P = (float)(kn / p->period);
        g.inv_P3 = (float)(1.0 / (p->period * p->period * p->period));

        double *radii = (double *)(base + oRadii);
        float *deconv = (float *)(base + oDeconv), *ballft = (float *)(base + oBallft);
        float2 *twn = (float2 *)(base + oTwn), *twN = (float2 *)(base + oTwN);
        float *consts = (float *)(base + oConsts);
        int *err = (int *)(base + oErr);
        int *boxes = (int *)(base + oBoxes);
        unsigned *stats = (unsigned *)(base + oStats);
        InstDesc *dinst = (InstDesc *)(base + oInst);
        PairDesc *dpairs = (PairDesc *)(base + oPairs);
        InstPlan *dplan = (InstPlan *)(base + oPlan);
        float4 *knots = (float4 *)(base + oKnots);
        float4 *ku = (float4 *)(base + oKu);
        float *grid = (float *)(base + oGrid);
        float2 *z1 = (float2 *)(base + oZ1), *y1 = (float2 *)(base + oY1), *h = (float2 *)(base + oH);

        // cleared every call: status words and the spreading boxes
        if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) != cudaSuccess) return ncuda(e, "clear err");
        if ((e = cudaMemsetAsync(stats, 0, sizeof(unsigned) * 4, st)) != cudaSuccess) return ncuda(e, "clear stats");
        if ((e = cudaMemsetAsync(grid, 0, kGridBytes, st)) != cudaSuccess) return ncuda(e, "clear grid");
        if ((e = launch_reset_boxes(boxes, 2, st)) != cudaSuccess) return ncuda(e, "reset boxes");
        // tables for this call's parameters
        if ((e = cudaMemcpyAsync(radii, p->level_radii, sizeof(double) * g.L, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return ncuda(e, "copy radii");
        if ((e = launch_build_tables(g, beta, p->period, radii, deconv, ballft, twn, twN, consts, st)) != cudaSuccess)
            return ncuda(e, "tables");
        // knots, with level and finiteness checks
        if (nA > 0 && (e = launch_pack_knots(xyzA, levelA, nA, g.L, knots, stats, st)) != cudaSuccess)
            return ncuda(e, "pack A");
        if (nB > 0 && (e = launch_pack_knots(xyzB, levelB, nB, g.L, knots + kK, stats + 2, st)) != cudaSuccess)
            return ncuda(e, "pack B");
        unsigned hs[4] = {0, 0, 0, 0};
        if ((e = cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return ncuda(e, "read checks");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ncuda(e, "sync");
        if ((hs[1] | hs[3]) & 1u) return nfail(BC_ERR_ARG, "bc_correlate_noalloc: level id out of range");
        if ((hs[1] | hs[3]) & 2u) return nfail(BC_ERR_ARG, "bc_correlate_noalloc: non-finite knot coordinate");

        // descriptors: A unrotated, B rotated by quat; every support box may span the whole period
        InstDesc inst[2];
        std::memset(inst, 0, sizeof(inst));
        const long long gstride = (long long)kL * kn * kn * kn, zstride = (long long)kL * kn * kn * kH,
                        ystride = (long long)kL * kn * kN * kH;
        for (int i = 0; i < 2; i++) {
            inst[i].knot_off = i == 0 ? 0 : nA;
            inst[i].nknots = i == 0 ? nA : nB;
            inst[i].src_off = 0;
            inst[i].cap_e = kn;
            inst[i].grid_off = i * gstride;
            inst[i].z1_off = i * zstride;
            inst[i].y1_off = i * ystride;
            inst[i].knots = knots + (i == 0 ? 0 : kK);
        }
        inst[0].q[0] = 1.f;
        for (int a = 0; a < 4; a++) inst[1].q[a] = quat[a];
        const PairDesc pr{0, 1, 0, 0, 0};
        if ((e = cudaMemcpyAsync(dinst, inst, sizeof(inst), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return ncuda(e, "copy descriptors");
        if ((e = cudaMemcpyAsync(dpairs, &pr, sizeof(pr), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return ncuda(e, "copy pair");

        Tables t{};
        t.deconv = deconv;
        t.ballft = ballft;
        t.tw_n = twn;
        t.tw_N = twN;
        t.qmax = kQ - 1;
        t.consts = consts;
        if ((e = launch_prepare(g, dinst, 2, nA > nB ? nA : nB, ku, boxes, dplan, err, nullptr, nullptr, st)) != cudaSuccess)
            return ncuda(e, "prepare");
        if ((e = launch_spread(g, t, dinst, nA + nB, ku, dplan, grid, nsm, st)) != cudaSuccess) return ncuda(e, "spread");
        if ((e = launch_fft_z(g, t, dinst, 2, dplan, grid, z1, nsm, st)) != cudaSuccess) return ncuda(e, "fft z");
        if ((e = launch_fft_y(g, t, dinst, 2, dplan, z1, y1, kn, nsm, st)) != cudaSuccess) return ncuda(e, "fft y");
        if ((e = launch_fft_x(g, t, dinst, dplan, dpairs, 1, y1, nullptr, nullptr, h, nsm, st)) != cudaSuccess)
            return ncuda(e, "fft x");
        if ((e = launch_ifft_y(g, t, dpairs, 1, h, nsm, st)) != cudaSuccess) return ncuda(e, "ifft y");
        if ((e = launch_ifft_z(g, t, dpairs, 1, h, out, nullptr, nsm, st)) != cudaSuccess) return ncuda(e, "ifft z");
        // the kernels' own status word: bit 0 = a support box beyond its capacity
        // (the instance was skipped), bit 8 = a bounded wait gave up
        int herr = 0;
        if ((e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return ncuda(e, "read status");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ncuda(e, "sync");
        if (herr & 256) return nfail(BC_ERR_TIMEOUT, "bc_correlate_noalloc: a device wait timed out");
        if (herr) return nfail(BC_ERR_INTERNAL, "bc_correlate_noalloc: a support box exceeded its capacity");
        return BC_OK;
    } catch (...) {
        return nfail(BC_ERR_INTERNAL, "bc_correlate_noalloc: unexpected exception");
    }
}
