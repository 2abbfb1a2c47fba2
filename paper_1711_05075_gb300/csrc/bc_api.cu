// C-ABI of the ball-union correlation library (declared in include/ballcorr.h).
//
// The context owns the FP64-built tables and every workspace; a correlation
// call fills instance/pair descriptors on the host, copies them to the device
// and enqueues the kernel sequence on the context stream.  Nothing here does
// arithmetic of the method: the host code sizes buffers, validates arguments
// and launches kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "../../include/ballcorr.h"
#include "bc_internal.h"

using namespace bc;

static thread_local std::string g_last_error;

void bc::set_last_error(const std::string &msg) { g_last_error = msg; }

static bc_status fail(bc_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

static bc_status cuda_fail(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? BC_ERR_OOM : BC_ERR_CUDA;
}

#define CK(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                              \
    } while (0)

namespace {

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need, bool zero, cudaStream_t s)
    {
        if (need <= bytes) return cudaSuccess;
        if (p) {
            cudaStreamSynchronize(s);
            cudaFree(p);
            p = nullptr;
            bytes = 0;
        }
        size_t cap = need + need / 4 + 256;
        cudaError_t e = cudaMalloc(&p, cap);
        if (e != cudaSuccess) return e;
        bytes = cap;
        if (zero) return cudaMemsetAsync(p, 0, cap, s);
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

// A page-locked host buffer that only grows (no copy may target it when it grows).
struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMallocHost(&p, need);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = need;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
};

// Device workspaces of one pipeline: the context's own, or a captured plan's.
struct Workspace {
    DevBuf ku, plan, inst, pairs, grid, z1, y1, h, fa, boxes, keys;
    DevBuf cnt, cur, rec;     // binned spreading: bin counts (kept zeroed), bin cursors, knot records
    DevBuf sync;              // work-queue and dependency counters of the persistent back-half launch
    bool grid_dirty = false;  // spreading boxes may hold values (an enqueue failed midway)
    bool boxes_dirty = true;  // support-box accumulators need their reset state
    bool bins_dirty = false;  // bin counts may be non-zero (an enqueue failed midway)
    std::vector<char> last_desc; // descriptors the device copies hold
    void *last_inst_p = nullptr, *last_pairs_p = nullptr;
    // passes recorded as CUDA graphs, by launch signature (least recently used
    // first out), and signatures seen once but not yet recorded
    struct Graph {
        std::vector<char> key;
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;
    };
    std::vector<Graph> graphs;
    std::vector<std::vector<char>> seen;
    unsigned long long tick = 0;
    void drop_graph()
    {
        for (Graph &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        graphs.clear();
        seen.clear();
    }
    void release()
    {
        drop_graph();
        DevBuf *b[] = {&ku, &plan, &inst, &pairs, &grid, &z1, &y1, &h, &fa, &boxes, &keys, &cnt, &cur, &rec, &sync};
        for (DevBuf *x : b) x->release();
        last_desc.clear();
        last_inst_p = last_pairs_p = nullptr;
    }
};

} // namespace

struct bc_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    // stream-ordered pool for the shapes' knot arrays and upload staging, keeping
    // its memory between uploads (the default pool hands it back at every
    // synchronisation, and mapping it again costs more than the upload itself)
    cudaMemPool_t pool = nullptr;
    int nsm = 1;
    Geometry g{};
    double beta = 0, period = 2.0;
    std::vector<double> radii;
    // tables
    double *radii_dev = nullptr;
    float *deconv = nullptr, *ballft = nullptr;
    float2 *tw_n = nullptr, *tw_N = nullptr;
    float *consts = nullptr; // [0] = exp(beta) / I0(beta), then the window's piecewise polynomials
    float *xw = nullptr;     // x-pass level weights (Tables::xw) of the correlation
    int *modes = nullptr;    // BC_MOMENTS lowest modes of the half spectrum, (m_x, m_y, m_z) each
    int qmax = 0;
    // device status word
    int *err_dev = nullptr;
    // page-locked words the host reads after a synchronisation: the status
    // word, and two per shape of a bc_shapes_create call
    int *pin = nullptr;
    PinBuf hstats;
    // implementation choices (bc_set_tuning / bc_autotune)
    int spread_mode = 0;  // 0: spreading boxes in HBM (k_spread + k_fft_z); 1: binned, fused into the z pass
    int sweep_batch = 64; // rotations per pass when a sweep's batch argument is 0
    int fft_sched = 0;    // alternative radix schedule per forward FP32 pass: bit 0 z, bit 1 y, bit 2 x
    int overlap = 1;      // passes after k_prepare launched as programmatic dependents
    int z_tc = 0;         // z pass as a DFT product on the tensor cores (spread 0; needs zdft)
    int persistent = 0;   // x, inverse-y and inverse-z passes as one persistent launch (bc_back.cu)
    float *zdft = nullptr; // its 32-cell DFT block, split TF32 (hi, then lo), FP32 contexts with N <= 128
    // workspaces
    Workspace ws;                 // pipeline workspaces of direct calls
    DevBuf outbuf, stats, learn, tune; // host-output staging, shape checks, learned-sweep and tuning scratch
    DevBuf score_ft;                   // shape-complementarity weights for (score_r0, score_lambda)
    DevBuf score_xw;                   // their x-pass level weights
    double score_r0 = -1.0, score_lambda = 0.0;
    std::set<bc_shape_s *> shapes; // live shapes; orphaned (device memory freed) by bc_destroy
    std::set<bc_mlp_s *> nets;     // live networks; orphaned the same way
    std::set<bc_query_s *> queries; // live single-configuration queries; orphaned the same way
    // profiling
    bool prof_on = false;
    int prof_max = 0, prof_calls = 0;
    long long prof_launches = 0;
    std::vector<cudaEvent_t> prof_ev; // prof_max x (BC_NUM_STAGES + 1)
    int last_ninst = 0, last_npairs = 0, last_mode = 0, last_back = 0, last_yz = 0;
    cudaStream_t capture_stream = nullptr; // private stream for recording graphs (the legacy stream cannot be captured)
    cudaEvent_t ev_a = nullptr, ev_b = nullptr; // orders a coarse context's stream with this one (bc_learned_sweep_coarse)
    bool replay = true;                    // repeated identical passes of direct calls replay a recorded graph
    std::vector<InstDesc> last_inst;
};

// A rotation sweep captured as one CUDA graph over its own workspaces.
struct bc_plan_s {
    bc_ctx_t ctx = nullptr;
    Workspace ws;
    DevBuf desc;               // every pass's instance and pair descriptors
    cudaGraphExec_t exec = nullptr;
    int k = 0;
    long long launches = 0;    // kernels per replay
};

struct bc_shape_s {
    bc_ctx_t ctx = nullptr;
    int n = 0;
    float4 *knots = nullptr;
    float rmax = 0.f;
};

// A configuration's truncated correlation spectrum (bc_query_create).
struct bc_query_s {
    bc_ctx_t ctx = nullptr;
    int count = 0;          // m'
    DevBuf modes, ghat, io; // int4 modes, their g^ values, staging for host points and results
    void release()
    {
        modes.release();
        ghat.release();
        io.release();
    }
};

cudaStream_t bc::ctx_stream(bc_ctx_s *c) { return c->stream; }
void bc::ctx_register_mlp(bc_ctx_s *c, bc_mlp_s *net) { c->nets.insert(net); }
void bc::ctx_unregister_mlp(bc_ctx_s *c, bc_mlp_s *net) { c->nets.erase(net); }
int *bc::ctx_err(bc_ctx_s *c) { return c->err_dev; }

static const char *kStageNames[BC_NUM_STAGES] = {"prepare", "spread", "fft_z", "fft_y", "fft_x", "ifft_y", "ifft_z"};

static void prof_free(bc_ctx_t c)
{
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_on = false;
    c->prof_max = c->prof_calls = 0;
    c->prof_launches = 0;
}

// Records the event that ends stage `stage` (-1 = start) of the current profiled call.
static void prof_mark(bc_ctx_t c, int stage)
{
    if (!c->prof_on || c->prof_calls >= c->prof_max) return;
    cudaEventRecord(c->prof_ev[(size_t)c->prof_calls * (BC_NUM_STAGES + 1) + (stage + 1)], c->stream);
}

static Tables tables_of(bc_ctx_t c)
{
    Tables t;
    t.deconv = c->deconv;
    t.ballft = c->ballft;
    t.tw_n = c->tw_n;
    t.tw_N = c->tw_N;
    t.qmax = c->qmax;
    t.consts = c->consts;
    t.xw = c->xw;
    return t;
}

// Per-axis capacity of an instance's support box: the stencil cells of knots
// with |u| <= U = rmax n / P span at most floor(2U) + W + 1 cells (the lowest
// cell is at least -U - W/2, the highest below U + W/2); one more cell covers
// the FP32 rounding of u (rmax is already rounded up).  Beyond n/2 the
// coordinates may wrap and the box is the whole period.  A box beyond its
// capacity raises the status word (bc_sync: BC_ERR_INTERNAL).
static int cap_extent(const bc_ctx_t c, float rmax)
{
    const double U = (double)rmax * c->g.n / c->period;
    if (U >= 0.5 * c->g.n - 1.0) return c->g.n;
    int e = (int)std::ceil(2.0 * U) + c->g.W + 2;
    return e > c->g.n ? c->g.n : e;
}

extern "C" {

const char *bc_last_error(void) { return g_last_error.c_str(); }

const char *bc_version(void) { return "ballcorr 0.1 (sm_103a, FP32 type-1 NUFFT correlation)"; }

bc_status bc_create(const bc_params *p, void *cuda_stream, bc_ctx_t *out)
{
    try {
        if (!p || !out) return fail(BC_ERR_ARG, "bc_create: null pointer");
        *out = nullptr;
        if (p->precision != 0 && p->precision != 1) return fail(BC_ERR_UNSUPPORTED, "bc_create: precision must be 0 or 1");
        if (p->precision == 1 && !supported_split(p->N))
            return fail(BC_ERR_UNSUPPORTED, "bc_create: precision 1 (split BF16) is built for N = 32, 64, 96, 128, 256");
        if (p->sigma != 2) return fail(BC_ERR_UNSUPPORTED, "bc_create: sigma must be 2");
        if (!supported_N(p->N)) return fail(BC_ERR_UNSUPPORTED, "bc_create: N must be one of 32, 64, 96, 128, 256");
        if (p->W < 2 || p->W > 10 || p->W > p->N) return fail(BC_ERR_ARG, "bc_create: W must be in [2, 10] and <= N");
        if (!(p->period > 0) || !std::isfinite(p->period)) return fail(BC_ERR_ARG, "bc_create: period must be > 0");
        if (p->level_count < 1 || p->level_count > BC_MAX_LEVELS)
            return fail(BC_ERR_ARG, "bc_create: level_count must be in [1, 8]");
        if (!p->level_radii) return fail(BC_ERR_ARG, "bc_create: level_radii is null");
        for (int l = 0; l < p->level_count; l++)
            if (!(p->level_radii[l] > 0) || !std::isfinite(p->level_radii[l]))
                return fail(BC_ERR_ARG, "bc_create: radii must be finite and > 0");
        double beta = p->beta;
        if (!(beta > 0)) {
            const double a = (double)p->W / p->sigma * (p->sigma - 0.5);
            beta = M_PI * std::sqrt(a * a - 0.8);
        }
        if (!std::isfinite(beta) || beta <= 0 || beta > 80) return fail(BC_ERR_ARG, "bc_create: beta out of range");
        // The spreading kernel evaluates the window with an FP32 beta; the FP64
        // deconvolution table must describe that same window.
        beta = (double)(float)beta;

        bc_ctx_t c = new (std::nothrow) bc_ctx_s();
        if (!c) return fail(BC_ERR_OOM, "bc_create: host allocation failed");
        c->stream = (cudaStream_t)cuda_stream;
        cudaError_t e0 = cudaGetDevice(&c->device);
        if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
        if (e0 != cudaSuccess) {
            delete c;
            return cuda_fail(e0, "bc_create: device query");
        }
        c->beta = beta;
        c->period = p->period;
        c->radii.assign(p->level_radii, p->level_radii + p->level_count);
        Geometry &g = c->g;
        g.N = p->N;
        g.n = p->sigma * p->N;
        g.W = p->W;
        g.L = p->level_count;
        g.H = p->N / 2;
        g.prec = p->precision;
        g.beta = (float)beta;
        g.n_over_P = (float)(g.n / p->period);
        g.inv_P3 = (float)(1.0 / (p->period * p->period * p->period));
        c->qmax = 3 * (g.N / 2) * (g.N / 2);
        auto bail = [&](cudaError_t e, const char *w) {
            bc_status s = cuda_fail(e, w);
            bc_destroy(c);
            return s;
        };
        cudaError_t e;
        if ((e = cudaMalloc(&c->radii_dev, sizeof(double) * g.L)) != cudaSuccess) return bail(e, "cudaMalloc radii");
        if ((e = cudaMalloc(&c->deconv, sizeof(float) * g.N)) != cudaSuccess) return bail(e, "cudaMalloc deconv");
        if ((e = cudaMalloc(&c->ballft, sizeof(float) * g.L * (c->qmax + 1))) != cudaSuccess) return bail(e, "cudaMalloc ballft");
        if ((e = cudaMalloc(&c->tw_n, sizeof(float2) * g.n)) != cudaSuccess) return bail(e, "cudaMalloc tw_n");
        if ((e = cudaMalloc(&c->tw_N, sizeof(float2) * g.N)) != cudaSuccess) return bail(e, "cudaMalloc tw_N");
        if ((e = cudaMalloc(&c->consts, sizeof(float) * CONSTS_FLOATS)) != cudaSuccess) return bail(e, "cudaMalloc consts");
        {
            // the BC_MOMENTS lowest modes of the half spectrum (m_z >= 0, m != 0, components
            // inside (-N/2, N/2)), ordered by (|m|^2, m_x, m_y, m_z)
            std::vector<std::array<int, 4>> all;
            const int h = g.N / 2;
            for (int mx = -h + 1; mx < h; mx++)
                for (int my = -h + 1; my < h; my++)
                    for (int mz = 0; mz < h; mz++)
                        if (mx || my || mz) all.push_back({mx * mx + my * my + mz * mz, mx, my, mz});
            std::sort(all.begin(), all.end());
            std::vector<int> tab(3 * BC_MOMENTS);
            for (int i = 0; i < BC_MOMENTS; i++)
                for (int j = 0; j < 3; j++) tab[3 * i + j] = all[i][1 + j];
            if (!moments_rot_table_matches(tab.data())) {
                bc_destroy(c);
                return fail(BC_ERR_INTERNAL, "bc_create: the compiled moment-mode table differs from the context's");
            }
            if ((e = cudaMalloc(&c->modes, sizeof(int) * tab.size())) != cudaSuccess) return bail(e, "cudaMalloc modes");
            if ((e = cudaMemcpy(c->modes, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
                return bail(e, "copy modes");
        }
        {
            cudaMemPoolProps pp{};
            pp.allocType = cudaMemAllocationTypePinned;
            pp.location.type = cudaMemLocationTypeDevice;
            pp.location.id = c->device;
            if ((e = cudaMemPoolCreate(&c->pool, &pp)) != cudaSuccess) return bail(e, "cudaMemPoolCreate");
            unsigned long long keep = ~0ull; // never trim at synchronisation (freed at bc_destroy)
            if ((e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
                return bail(e, "pool release threshold");
        }
        if ((e = cudaMalloc(&c->err_dev, sizeof(int))) != cudaSuccess) return bail(e, "cudaMalloc err");
        if ((e = cudaMallocHost(&c->pin, sizeof(int))) != cudaSuccess) return bail(e, "cudaMallocHost");
        *c->pin = 0;
        if ((e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream)) != cudaSuccess) return bail(e, "memset err");
        if ((e = cudaMemcpyAsync(c->radii_dev, c->radii.data(), sizeof(double) * g.L, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return bail(e, "copy radii");
        if ((e = launch_build_tables(g, beta, p->period, c->radii_dev, c->deconv, c->ballft, c->tw_n, c->tw_N, c->consts, c->stream)) != cudaSuccess)
            return bail(e, "build tables");
        if ((e = cudaMalloc(&c->xw, sizeof(float) * xw_floats(g))) != cudaSuccess) return bail(e, "cudaMalloc xw");
        if ((e = launch_build_xw(g, c->deconv, c->ballft, c->xw, c->stream)) != cudaSuccess) return bail(e, "build x weights");
        if (g.prec == 0 && g.n == 2 * g.N && supported_z_umma(g.N)) {
            const size_t half = (size_t)(g.n / 2) * 32;
            if ((e = cudaMalloc(&c->zdft, sizeof(float) * 2 * half)) != cudaSuccess) return bail(e, "cudaMalloc zdft");
            if ((e = launch_build_zdft(g.n, c->zdft, c->zdft + half, c->stream)) != cudaSuccess) return bail(e, "build zdft");
            c->z_tc = 1;
        }
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e, "bc_create sync");
        *out = c;
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_create: unexpected exception");
    }
}

bc_status bc_destroy(bc_ctx_t c)
{
    if (!c) return BC_OK;
    try {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->radii_dev);
        cudaFree(c->deconv);
        cudaFree(c->ballft);
        cudaFree(c->tw_n);
        cudaFree(c->tw_N);
        cudaFree(c->xw);
        cudaFree(c->err_dev);
        if (c->pin) cudaFreeHost(c->pin);
        cudaFree(c->consts);
        cudaFree(c->modes);
        cudaFree(c->zdft);
        prof_free(c);
        for (bc_shape_s *s : c->shapes) {
            if (s->knots) cudaFreeAsync(s->knots, c->stream);
            s->knots = nullptr;
            s->ctx = nullptr;
        }
        c->shapes.clear();
        cudaStreamSynchronize(c->stream);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        for (bc_mlp_s *net : c->nets) mlp_orphan(net);
        c->nets.clear();
        for (bc_query_s *q : c->queries) {
            q->release();
            q->ctx = nullptr;
        }
        c->queries.clear();
        c->ws.release();
        if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
        if (c->ev_a) cudaEventDestroy(c->ev_a);
        if (c->ev_b) cudaEventDestroy(c->ev_b);
        DevBuf *bufs[] = {&c->outbuf, &c->stats, &c->learn, &c->tune, &c->score_ft, &c->score_xw};
        for (DevBuf *b : bufs) b->release();
        c->hstats.release();
        delete c;
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_destroy: unexpected exception");
    }
}

// The device address of a page-locked host buffer mapped into the device
// address space (cudaMallocHost, cudaHostAlloc, cudaHostRegister), through
// which kernels read or write it directly; null for any other host memory.
static void *mapped_host_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

bc_status bc_shapes_create(bc_ctx_t c, int count, const float *const *xyz, const int *const *level, const int *n,
                           int on_device, bc_shape_t *out)
{
    try {
        if (!c || !out || count < 0 || (count > 0 && (!xyz || !level || !n)))
            return fail(BC_ERR_ARG, "bc_shapes_create: null argument or count < 0");
        for (int i = 0; i < count; i++) out[i] = nullptr;
        // Host arrays in mapped page-locked memory are read by the packing kernel
        // through their device addresses; other host arrays are copied to a device
        // staging area first.
        std::vector<const float *> mx(count, nullptr);
        std::vector<const int *> ml(count, nullptr);
        size_t staged = 0; // staging bytes of the host-resident shapes that are not mapped
        for (int i = 0; i < count; i++) {
            const std::string who = "bc_shape_create (shape " + std::to_string(i) + "): ";
            if (n[i] < 0) return fail(BC_ERR_ARG, who + "n < 0");
            if (n[i] > 0 && (!xyz[i] || !level[i])) return fail(BC_ERR_ARG, who + "null knot arrays");
            if (n[i] >= (1 << 26)) return fail(BC_ERR_ARG, who + "too many knots");
            if (!on_device && n[i] > 0) {
                mx[i] = (const float *)mapped_host_ptr(xyz[i]);
                ml[i] = (const int *)mapped_host_ptr(level[i]);
                if (!mx[i] || !ml[i]) {
                    mx[i] = nullptr;
                    ml[i] = nullptr;
                    staged += (sizeof(float) * 3 + sizeof(int)) * (size_t)n[i];
                }
            }
        }
        std::vector<bc_shape_t> made(count, nullptr);
        cudaStream_t st = c->stream;
        void *staging = nullptr;
        auto drop = [&]() {
            // queued copies and packing kernels may still read the caller's arrays
            cudaStreamSynchronize(st);
            if (staging) cudaFreeAsync(staging, st);
            for (bc_shape_t s : made)
                if (s) {
                    if (s->knots) cudaFreeAsync(s->knots, st);
                    delete s;
                }
        };
        auto bail = [&](cudaError_t e, const char *w) {
            bc_status r = cuda_fail(e, w);
            drop();
            return r;
        };
        for (int i = 0; i < count; i++) {
            made[i] = new (std::nothrow) bc_shape_s();
            if (!made[i]) {
                drop();
                return fail(BC_ERR_OOM, "bc_shape_create: host allocation failed");
            }
            made[i]->ctx = c;
            made[i]->n = n[i];
        }
        cudaError_t e;
        if (staged && (e = cudaMallocFromPoolAsync(&staging, staged, c->pool, st)) != cudaSuccess)
            return bail(e, "cudaMallocAsync staging");
        if ((e = c->stats.ensure(2 * sizeof(unsigned int) * (size_t)(count > 0 ? count : 1), false, st)) != cudaSuccess)
            return bail(e, "stats");
        if ((e = c->hstats.ensure(2 * sizeof(unsigned int) * (size_t)(count > 0 ? count : 1))) != cudaSuccess)
            return bail(e, "page-locked stats");
        unsigned int *stats = (unsigned int *)c->stats.p;
        if (count && (e = cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned int) * count, st)) != cudaSuccess)
            return bail(e, "memset stats");
        char *sp = (char *)staging;
        for (int i = 0; i < count; i++) {
            const int ni = n[i];
            if (ni == 0) continue;
            bc_shape_t s = made[i];
            if ((e = cudaMallocFromPoolAsync((void **)&s->knots, sizeof(float4) * ni, c->pool, st)) != cudaSuccess)
                return bail(e, "cudaMallocAsync knots");
            const float *dx = xyz[i];
            const int *dl = level[i];
            if (mx[i]) {
                dx = mx[i];
                dl = ml[i];
            } else if (!on_device) {
                float *sx = (float *)sp;
                int *sl = (int *)(sx + 3 * (size_t)ni);
                sp += (sizeof(float) * 3 + sizeof(int)) * (size_t)ni;
                if ((e = cudaMemcpyAsync(sx, dx, sizeof(float) * 3 * ni, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                    return bail(e, "copy xyz");
                if ((e = cudaMemcpyAsync(sl, dl, sizeof(int) * ni, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                    return bail(e, "copy level");
                dx = sx;
                dl = sl;
            }
            if ((e = launch_pack_knots(dx, dl, ni, c->g.L, s->knots, stats + 2 * i, st)) != cudaSuccess)
                return bail(e, "pack knots");
        }
        // one read-back through page-locked memory and one stream synchronisation
        // for every shape of the call
        unsigned int *hs = (unsigned int *)c->hstats.p;
        if (count && (e = cudaMemcpyAsync(hs, stats, 2 * sizeof(unsigned int) * count, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return bail(e, "copy stats");
        if (staging) {
            e = cudaFreeAsync(staging, st);
            staging = nullptr;
            if (e != cudaSuccess) return bail(e, "free staging");
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "bc_shape_create sync");
        for (int i = 0; i < count; i++) {
            if (n[i] == 0) continue;
            const std::string who = "bc_shape_create (shape " + std::to_string(i) + "): ";
            if (hs[2 * i + 1] & 1u) {
                drop();
                return fail(BC_ERR_ARG, who + "level id out of range [0, L)");
            }
            if (hs[2 * i + 1] & 2u) {
                drop();
                return fail(BC_ERR_ARG, who + "non-finite knot coordinate");
            }
            float r2;
            std::memcpy(&r2, &hs[2 * i], sizeof(float));
            made[i]->rmax = std::sqrt(r2) * (1.0f + 1e-6f);
        }
        for (int i = 0; i < count; i++) {
            c->shapes.insert(made[i]);
            out[i] = made[i];
        }
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_shape_create: unexpected exception");
    }
}

bc_status bc_shape_create(bc_ctx_t c, const float *xyz, const int *level, int n, int on_device, bc_shape_t *out)
{
    if (!out) return fail(BC_ERR_ARG, "bc_shape_create: null output");
    return bc_shapes_create(c, 1, &xyz, &level, &n, on_device, out);
}

bc_status bc_shape_destroy(bc_shape_t s)
{
    if (!s) return BC_OK;
    try {
        if (s->ctx) { // not orphaned by bc_destroy
            if (s->knots) cudaFreeAsync(s->knots, s->ctx->stream);
            s->ctx->shapes.erase(s);
        }
        delete s;
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_shape_destroy: unexpected exception");
    }
}

bc_status bc_sync(bc_ctx_t c)
{
    if (!c) return fail(BC_ERR_ARG, "bc_sync: null context");
    CK(cudaMemcpyAsync(c->pin, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int herr = c->pin[0];
    if (herr) {
        CK(cudaMemset(c->err_dev, 0, sizeof(int)));
        if (herr & 4) return fail(BC_ERR_ARG, "a device-resident rotation had zero norm");
        if (herr & 8)
            return fail(BC_ERR_TIMEOUT, "the tensor-core z transform stalled (a bounded wait expired); results are incomplete");
        if (herr & 16)
            return fail(BC_ERR_TIMEOUT, "a dependency wait of the persistent launch expired; results are incomplete");
        if (herr & 32)
            return fail(BC_ERR_TIMEOUT, "a tensor-core product of the MLP stalled (a bounded wait expired); results are incomplete");
        return fail(BC_ERR_INTERNAL, "device-side check failed (support box exceeded its capacity)");
    }
    return BC_OK;
}

bc_status bc_selftest_wait(bc_ctx_t c)
{
    if (!c) return fail(BC_ERR_ARG, "bc_selftest_wait: null context");
    CK(cudaStreamSynchronize(c->stream));
    if (c->ws.sync.ensure(sizeof(unsigned), false, c->stream) != cudaSuccess)
        return fail(BC_ERR_OOM, "bc_selftest_wait: counter");
    CK(launch_wait_selftest(c->err_dev, c->stream));
    CK(launch_queue_wait_selftest((unsigned *)c->ws.sync.p, c->err_dev, c->stream));
    CK(cudaMemcpyAsync(c->pin, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int herr = c->pin[0];
    CK(cudaMemset(c->err_dev, 0, sizeof(int)));
    if ((herr & 8) && (herr & 16))
        return fail(BC_ERR_TIMEOUT, "both self-test waits expired and reported it (the tensor-core mbarrier wait and "
                                    "the persistent launch's dependency wait)");
    return fail(BC_ERR_INTERNAL, "a self-test wait did not report its expiry");
}

const char *bc_stage_name(int i) { return (i >= 0 && i < BC_NUM_STAGES) ? kStageNames[i] : ""; }

bc_status bc_profile_begin(bc_ctx_t c, int max_calls)
{
    if (!c || max_calls < 1 || max_calls > (1 << 16)) return fail(BC_ERR_ARG, "bc_profile_begin: bad arguments");
    CK(cudaStreamSynchronize(c->stream));
    prof_free(c);
    c->prof_ev.resize((size_t)max_calls * (BC_NUM_STAGES + 1));
    for (auto &ev : c->prof_ev) CK(cudaEventCreate(&ev));
    c->prof_max = max_calls;
    c->prof_on = true;
    return BC_OK;
}

bc_status bc_profile_end(bc_ctx_t c, bc_profile *out)
{
    if (!c || !out) return fail(BC_ERR_ARG, "bc_profile_end: null argument");
    if (!c->prof_on) return fail(BC_ERR_ARG, "bc_profile_end: bc_profile_begin was not called");
    std::memset(out, 0, sizeof(*out));
    CK(cudaStreamSynchronize(c->stream));
    out->calls = c->prof_calls;
    out->launches = c->prof_launches;
    for (int k = 0; k < c->prof_calls; k++) {
        for (int s = 0; s < BC_NUM_STAGES; s++) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->prof_ev[(size_t)k * (BC_NUM_STAGES + 1) + s],
                                    c->prof_ev[(size_t)k * (BC_NUM_STAGES + 1) + s + 1]));
            out->ms[s] += ms;
        }
    }
    // algorithmic bytes of the last call, from its device plan
    if (c->prof_calls > 0 && c->last_ninst > 0) {
        std::vector<InstPlan> pl(c->last_ninst);
        CK(cudaMemcpy(pl.data(), c->ws.plan.p, sizeof(InstPlan) * c->last_ninst, cudaMemcpyDeviceToHost));
        const double L = c->g.L, N = c->g.N, H = c->g.H;
        double knots = 0, cells = 0, zc = 0, yc = 0;
        for (int i = 0; i < c->last_ninst; i++) {
            const double b0 = pl[i].b[0], b1 = pl[i].b[1], b2 = pl[i].b[2];
            knots += c->last_inst[i].nknots;
            cells += L * b0 * b1 * b2;   // spreading boxes
            zc += L * b0 * b1 * H;       // z-transformed rows
            yc += L * b0 * N * H;        // y-transformed planes
        }
        const double P = c->last_npairs, half = N * N * H;
        out->bytes[0] = knots * 16.0 * 2.0;                 // knots in, prepared knots out
        if (c->last_mode == 1) {
            out->bytes[1] = knots * (16.0 + 4.0 * BIN_REC); // prepared knots in, binned records out
            out->bytes[2] = knots * 4.0 * BIN_REC + zc * 8.0; // records in (once), z rows out
        } else {
            out->bytes[1] = knots * 16.0 + cells * 4.0;     // prepared knots in, boxes out
            out->bytes[2] = cells * 4.0 + zc * 8.0;
        }
        out->bytes[3] = zc * 8.0 + yc * 8.0;
        out->bytes[4] = yc * 8.0 + P * half * 8.0;
        out->bytes[5] = 2.0 * P * half * 8.0;
        out->bytes[6] = P * half * 8.0 + P * N * N * N * 4.0;
        if (c->last_back) { // one persistent launch carried the three passes
            out->bytes[4] += out->bytes[5] + out->bytes[6];
            out->bytes[5] = out->bytes[6] = 0.0;
        } else if (c->last_yz) { // planes read once, grids written once
            out->bytes[5] = 0.0;
        }
    }
    prof_free(c);
    return BC_OK;
}

} // extern "C"

// One pass of the pipeline over `shapes` (instance i is shapes[i] rotated by
// quats[i], identity when null, or by the device quaternion qdev[i]) and
// `pairs`.  With cache_first, pairs[0] = (a, -1) writes instance a's spectrum
// into the workspace's cache and the remaining pairs follow; pairs with
// a = -1 read that cache.
// Per-level multiplier of the spectra and the sign of the product: the ball
// transforms for a correlation; the complementarity weights, negated, for a
// score.
struct Weights {
    const float *ballft = nullptr; // null: the context's ball transform table
    const float *xw = nullptr;     // x-pass level weights built from ballft
    float sign = 1.f;
};

struct Job {
    std::vector<InstDesc> inst;
    std::vector<PairDesc> pairs;
    bool cache_first = false;
    int mode = 0;  // spreading: 0 boxes in HBM, 1 binned (fused into the z pass)
    int sched = 0; // radix schedule of the forward passes
    int ztc = 0;   // z pass on the tensor cores (mode 0 only)
    int back = 0;  // x, inverse-y and inverse-z passes as one persistent launch
    int overlap = 0; // passes after k_prepare as programmatic dependents of the pass before
    bool yz = false; // inverse y and z of whole planes in one launch (batches of many pairs)
    Weights w;
    int nmain = 0, koff = 0, max_knots = 0, max_cap = 0;
    long long goff = 0, zoff = 0, yoff = 0, hpairs = 0;
};

static Job plan_job(bc_ctx_t c, const std::vector<bc_shape_t> &shapes, const std::vector<const float *> &quats,
                    const std::vector<PairDesc> &pairs, bool cache_first, const std::vector<const float *> *qdev)
{
    const Geometry &g = c->g;
    const int N = g.N, H = g.H, L = g.L;
    Job j;
    j.pairs = pairs;
    j.cache_first = cache_first;
    j.mode = c->spread_mode;
    j.sched = c->fft_sched;
    j.ztc = c->z_tc && c->spread_mode == 0 ? 1 : 0;
    j.back = c->persistent;
    j.overlap = c->overlap;
    j.nmain = (int)pairs.size() - (cache_first ? 1 : 0);
    j.inst.resize(shapes.size());
    for (size_t i = 0; i < shapes.size(); i++) {
        bc_shape_t s = shapes[i];
        InstDesc &d = j.inst[i];
        std::memset(&d, 0, sizeof(d));
        d.knot_off = j.koff;
        d.nknots = s->n;
        d.src_off = 0;
        d.knots = s->knots;
        const int e = cap_extent(c, s->rmax);
        d.cap_e = e;
        j.max_cap = std::max(j.max_cap, e);
        d.grid_off = j.goff;
        d.z1_off = j.zoff;
        d.y1_off = j.yoff;
        if (quats[i]) {
            for (int q = 0; q < 4; q++) d.q[q] = quats[i][q];
        } else {
            d.q[0] = 1.f;
        }
        if (qdev) d.qdev = (*qdev)[i];
        j.koff += s->n;
        j.max_knots = std::max(j.max_knots, s->n);
        j.goff += (long long)L * e * (((e + 31) / 32) * 32) * e; // block-transposed boxes, y padded to 32
        j.zoff += (long long)L * e * e * H;
        j.yoff += (long long)L * e * N * H;
    }
    for (const PairDesc &p : pairs)
        if (p.b >= 0) j.hpairs = std::max(j.hpairs, p.h_off / ((long long)N * N * H) + 1);
    // plane-wise inverse passes once there are enough planes to fill the device
    // (one block each, two per SM) several times over
    j.yz = !j.back && g.N <= 128 && (long long)j.nmain * N >= 4LL * 2 * c->nsm;
    return j;
}

// Grows the workspace to hold passes of up to these sizes (may synchronise the
// stream and allocate; never called while a stream is being captured).
static bc_status ensure_ws(bc_ctx_t c, Workspace &ws, int mode, long long koff, long long ninst, long long npairs,
                           long long goff, long long zoff, long long yoff, long long hpairs)
{
    cudaStream_t st = c->stream;
    const int N = c->g.N, H = c->g.H;
    cudaError_t e;
    if (mode == 1) {
        goff = 1; // no spreading boxes
        const size_t nbins = (size_t)std::max(ninst, 1LL) * c->g.L * c->g.n;
        const size_t before = ws.cnt.bytes;
        if ((e = ws.cnt.ensure(sizeof(int) * nbins, true, st)) != cudaSuccess) return cuda_fail(e, "bin counts");
        if (ws.bins_dirty && ws.cnt.bytes == before) {
            if ((e = cudaMemsetAsync(ws.cnt.p, 0, ws.cnt.bytes, st)) != cudaSuccess) return cuda_fail(e, "bin counts clear");
        }
        ws.bins_dirty = false;
        if ((e = ws.cur.ensure(sizeof(int) * nbins, false, st)) != cudaSuccess) return cuda_fail(e, "bin cursors");
        if ((e = ws.rec.ensure(sizeof(float) * BIN_REC * (size_t)std::max(koff, 1LL), false, st)) != cudaSuccess)
            return cuda_fail(e, "knot records");
    }
    if ((e = ws.ku.ensure(sizeof(float4) * (size_t)std::max(koff, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "ku");
    if ((e = ws.plan.ensure(sizeof(InstPlan) * (size_t)std::max(ninst, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "plan");
    {
        const size_t before = ws.boxes.bytes;
        if ((e = ws.boxes.ensure(sizeof(int) * 8 * (size_t)std::max(ninst, 1LL), false, st)) != cudaSuccess)
            return cuda_fail(e, "boxes");
        if (ws.boxes.bytes != before || ws.boxes_dirty) {
            if ((e = launch_reset_boxes((int *)ws.boxes.p, (int)(ws.boxes.bytes / (8 * sizeof(int))), st)) != cudaSuccess)
                return cuda_fail(e, "reset boxes");
            ws.boxes_dirty = false;
        }
    }
    if ((e = ws.inst.ensure(sizeof(InstDesc) * (size_t)std::max(ninst, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "inst");
    if ((e = ws.pairs.ensure(sizeof(PairDesc) * (size_t)std::max(npairs, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "pairs");
    const size_t grid_before = ws.grid.bytes;
    if ((e = ws.grid.ensure(sizeof(float) * (size_t)std::max(goff, 1LL), true, st)) != cudaSuccess) return cuda_fail(e, "grid");
    if (ws.grid_dirty && ws.grid.bytes == grid_before) {
        if ((e = cudaMemsetAsync(ws.grid.p, 0, ws.grid.bytes, st)) != cudaSuccess) return cuda_fail(e, "grid clear");
    }
    ws.grid_dirty = false;
    if ((e = ws.z1.ensure(sizeof(float2) * (size_t)std::max(zoff, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "z1");
    if ((e = ws.y1.ensure(sizeof(float2) * (size_t)std::max(yoff, 1LL), false, st)) != cudaSuccess) return cuda_fail(e, "y1");
    if (hpairs > 0 && (e = ws.h.ensure(sizeof(float2) * (size_t)hpairs * N * N * H, false, st)) != cudaSuccess)
        return cuda_fail(e, "h");
    if ((e = ws.fa.ensure(sizeof(float2) * (size_t)N * N * H, false, st)) != cudaSuccess) return cuda_fail(e, "fa");
    if ((e = ws.sync.ensure(sizeof(unsigned) * back_sync_words(N, (int)std::max(npairs, 1LL)), false, st)) != cudaSuccess)
        return cuda_fail(e, "queue counters");
    return BC_OK;
}

// The kernel launches of one planned pass, with its descriptors already on the
// device at dinst / dpairs.  Launches only (legal while a stream is captured).
static bc_status launch_job(bc_ctx_t c, Workspace &ws, const Job &job, const InstDesc *dinst, const PairDesc *dpairs,
                            float *dout, unsigned long long *keys, bool profile, cudaStream_t st,
                            long long *nlaunch = nullptr)
{
    Geometry g = c->g;
    g.inv_P3 *= job.w.sign;
    g.sched = job.sched;
    g.pdl = job.overlap;
    const int ninst = (int)job.inst.size();
    Tables t = tables_of(c);
    if (job.w.ballft) {
        t.ballft = job.w.ballft;
        t.xw = job.w.xw;
    }
    InstPlan *dplan = (InstPlan *)ws.plan.p;
    const PairDesc *pmain = dpairs + (job.cache_first ? 1 : 0);
    const int nmain = job.nmain;
    cudaError_t e;
    int launches = 0;
    const bool prof = profile && c->prof_on && c->prof_calls < c->prof_max;
    auto mark = [&](int s) {
        if (profile) prof_mark(c, s);
    };
    const bool binned = job.mode == 1;
    mark(-1);
    ws.boxes_dirty = true; // until the plan has consumed and reset the accumulators
    if (binned) {
        ws.bins_dirty = true; // until the bin scan has consumed and cleared the counts
        if ((e = launch_prepare(g, dinst, ninst, job.max_knots, (float4 *)ws.ku.p, (int *)ws.boxes.p, dplan,
                                c->err_dev, (int *)ws.cnt.p, (int *)ws.cur.p, st)) != cudaSuccess)
            return cuda_fail(e, "prepare");
        ws.bins_dirty = false;
        launches += 2;
    } else {
        ws.grid_dirty = true; // until the z pass has consumed the spreading boxes
        if ((e = launch_prepare(g, dinst, ninst, job.max_knots, (float4 *)ws.ku.p, (int *)ws.boxes.p, dplan,
                                c->err_dev, nullptr, nullptr, st)) != cudaSuccess)
            return cuda_fail(e, "prepare");
        launches += 1;
    }
    ws.boxes_dirty = false;
    mark(0);
    if (binned) {
        if ((e = launch_bin(g, t, dinst, job.koff, (const float4 *)ws.ku.p, dplan, (int *)ws.cur.p, (float *)ws.rec.p, st)) != cudaSuccess)
            return cuda_fail(e, "bin");
    } else {
        if ((e = launch_spread(g, t, dinst, job.koff, (const float4 *)ws.ku.p, dplan, (float *)ws.grid.p, c->nsm, st)) != cudaSuccess)
            return cuda_fail(e, "spread");
    }
    launches += job.koff > 0;
    mark(1);
    if (binned) {
        if ((e = launch_fft_z_binned(g, t, dinst, ninst, dplan, (const int *)ws.cur.p, (const float *)ws.rec.p,
                                     (float2 *)ws.z1.p, c->nsm, st)) != cudaSuccess)
            return cuda_fail(e, "fft z (binned)");
    } else {
        if (job.ztc) {
            const size_t half = (size_t)(g.n / 2) * 32;
            if ((e = launch_fft_z_umma(g, t, dinst, ninst, dplan, (float *)ws.grid.p, (float2 *)ws.z1.p, c->zdft,
                                       c->zdft + half, c->err_dev, c->nsm, st)) != cudaSuccess)
                return cuda_fail(e, "fft z (tensor cores)");
        } else if ((e = launch_fft_z(g, t, dinst, ninst, dplan, (float *)ws.grid.p, (float2 *)ws.z1.p, c->nsm, st)) != cudaSuccess) {
            return cuda_fail(e, "fft z");
        }
        ws.grid_dirty = false;
    }
    launches++;
    mark(2);
    if ((e = launch_fft_y(g, t, dinst, ninst, dplan, (const float2 *)ws.z1.p, (float2 *)ws.y1.p, job.max_cap, c->nsm,
                          st)) != cudaSuccess)
        return cuda_fail(e, "fft y");
    launches++;
    mark(3);
    if (job.cache_first) {
        if ((e = launch_fft_x(g, t, dinst, dplan, dpairs, 1, (const float2 *)ws.y1.p, nullptr, (float2 *)ws.fa.p,
                              (float2 *)ws.h.p, c->nsm, st)) != cudaSuccess)
            return cuda_fail(e, "fft x (cache)");
        launches++;
    }
    if (job.back && nmain > 0) {
        // one persistent launch for the three passes; profiled, its time is
        // the fft_x stage and the two inverse stages read zero
        if ((e = launch_back(g, t, dinst, dplan, pmain, nmain, (const float2 *)ws.y1.p, (const float2 *)ws.fa.p,
                             (float2 *)ws.h.p, dout, keys, (unsigned *)ws.sync.p, c->err_dev, c->nsm, st)) != cudaSuccess)
            return cuda_fail(e, "persistent back half");
        launches++;
        mark(4);
        mark(5);
        mark(6);
    } else {
        if (nmain > 0) {
            if ((e = launch_fft_x(g, t, dinst, dplan, pmain, nmain, (const float2 *)ws.y1.p, (const float2 *)ws.fa.p,
                                  nullptr, (float2 *)ws.h.p, c->nsm, st)) != cudaSuccess)
                return cuda_fail(e, "fft x");
            launches++;
        }
        mark(4);
        if (job.yz) {
            // many pairs: both inverse passes plane by plane in shared memory (one
            // launch, timed as the ifft_z stage)
            mark(5);
            if ((e = launch_ifft_yz(g, t, pmain, nmain, (const float2 *)ws.h.p, dout, keys, c->nsm, st)) != cudaSuccess)
                return cuda_fail(e, "ifft yz");
            launches++;
        } else {
            if (nmain > 0) {
                if ((e = launch_ifft_y(g, t, pmain, nmain, (float2 *)ws.h.p, c->nsm, st)) != cudaSuccess)
                    return cuda_fail(e, "ifft y");
                launches++;
            }
            mark(5);
            if (nmain > 0) {
                if ((e = launch_ifft_z(g, t, pmain, nmain, (const float2 *)ws.h.p, dout, keys, c->nsm, st)) != cudaSuccess)
                    return cuda_fail(e, "ifft z");
                launches++;
            }
        }
        mark(6);
    }
    if (nlaunch) *nlaunch += launches;
    if (prof) {
        c->prof_calls++;
        c->prof_launches += launches;
        c->last_ninst = ninst;
        c->last_npairs = nmain;
        c->last_mode = job.mode;
        c->last_back = job.back && nmain > 0;
        c->last_yz = job.yz;
        c->last_inst = job.inst;
    }
    return BC_OK;
}

// Plans, uploads the descriptors (only when they changed) and launches one pass
// on the context's own workspace.
static bc_status enqueue(bc_ctx_t c, const std::vector<bc_shape_t> &shapes, const std::vector<const float *> &quats,
                         const std::vector<PairDesc> &pairs, bool cache_first, float *dout, unsigned long long *keys,
                         const std::vector<const float *> *qdev = nullptr, Weights w = Weights())
{
    Workspace &ws = c->ws;
    Job job = plan_job(c, shapes, quats, pairs, cache_first, qdev);
    job.w = w;
    const long long ninst = (long long)job.inst.size(), npairs = (long long)job.pairs.size();
    if (bc_status s = ensure_ws(c, ws, job.mode, job.koff, ninst, npairs, job.goff, job.zoff, job.yoff, job.hpairs)) return s;
    const size_t inst_bytes = sizeof(InstDesc) * ninst, pair_bytes = sizeof(PairDesc) * npairs;
    std::vector<char> desc(inst_bytes + pair_bytes);
    std::memcpy(desc.data(), job.inst.data(), inst_bytes);
    std::memcpy(desc.data() + inst_bytes, job.pairs.data(), pair_bytes);
    if (desc != ws.last_desc || ws.inst.p != ws.last_inst_p || ws.pairs.p != ws.last_pairs_p) {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(ws.inst.p, desc.data(), inst_bytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(e, "copy inst");
        if ((e = cudaMemcpyAsync(ws.pairs.p, desc.data() + inst_bytes, pair_bytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(e, "copy pairs");
        ws.last_desc.swap(desc);
        ws.last_inst_p = ws.inst.p;
        ws.last_pairs_p = ws.pairs.p;
    }
    const bool profiling = c->prof_on && c->prof_calls < c->prof_max;
    if (profiling || !c->replay)
        return launch_job(c, ws, job, (const InstDesc *)ws.inst.p, (const PairDesc *)ws.pairs.p, dout, keys, true, c->stream);
    // Replay.  The kernels read the instance and pair descriptors from device
    // memory, so two passes with the same launch signature -- counts and sizes
    // that set grids and kernel arguments, output and workspace buffers,
    // weights, spreading implementation -- are the same launches, whatever the
    // descriptors hold.  A signature is recorded as a graph when it is seen the
    // second time, and replayed from then on.
    std::vector<char> key;
    auto add = [&](const void *v, size_t n) { key.insert(key.end(), (const char *)v, (const char *)v + n); };
    const long long sig[] = {(long long)job.inst.size(), (long long)job.pairs.size(), (long long)job.nmain,
                             (long long)job.cache_first, (long long)job.koff, (long long)job.max_knots,
                             (long long)job.mode, (long long)job.sched, (long long)job.ztc, (long long)job.back,
                             (long long)job.max_cap, (long long)job.overlap};
    add(sig, sizeof(sig));
    const void *ptrs[] = {dout, keys, job.w.ballft, ws.ku.p, ws.plan.p, ws.inst.p, ws.pairs.p, ws.grid.p, ws.z1.p, ws.y1.p,
                          ws.h.p, ws.fa.p, ws.boxes.p, ws.cnt.p, ws.cur.p, ws.rec.p, ws.sync.p, c->stream};
    add(ptrs, sizeof(ptrs));
    add(&job.w.sign, sizeof(job.w.sign));
    constexpr size_t kMaxGraphs = 8;
    cudaError_t e;
    Workspace::Graph *hit = nullptr;
    for (Workspace::Graph &g : ws.graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        auto it = std::find(ws.seen.begin(), ws.seen.end(), key);
        if (it == ws.seen.end()) { // first sighting: launch kernel by kernel
            if (ws.seen.size() >= kMaxGraphs) ws.seen.erase(ws.seen.begin());
            ws.seen.push_back(key);
            return launch_job(c, ws, job, (const InstDesc *)ws.inst.p, (const PairDesc *)ws.pairs.p, dout, keys, true,
                              c->stream);
        }
        ws.seen.erase(it);
        if (!c->capture_stream && (e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "capture stream");
        if ((e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
            return cuda_fail(e, "begin capture");
        bc_status s = launch_job(c, ws, job, (const InstDesc *)ws.inst.p, (const PairDesc *)ws.pairs.p, dout, keys, false,
                                 c->capture_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->capture_stream, &graph);
        if (s == BC_OK && e != cudaSuccess) s = cuda_fail(e, "end capture");
        cudaGraphExec_t exec = nullptr;
        if (s == BC_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) s = cuda_fail(e, "instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (s != BC_OK) return s;
        if (ws.graphs.size() >= kMaxGraphs) { // evict the least recently used
            auto lru = std::min_element(ws.graphs.begin(), ws.graphs.end(),
                                        [](const Workspace::Graph &x, const Workspace::Graph &y) { return x.used < y.used; });
            cudaGraphExecDestroy(lru->exec);
            ws.graphs.erase(lru);
        }
        ws.graphs.push_back(Workspace::Graph{std::move(key), exec, 0});
        hit = &ws.graphs.back();
    }
    hit->used = ++ws.tick;
    if ((e = cudaGraphLaunch(hit->exec, c->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    return BC_OK;
}

// Peaks for k rotations of B (host quaternions qhost, or device quaternions
// qdev) against A: A's spectrum once into the cache, then batches of
// rotations folded into peak keys, then keys -> peak / argmax.
static bc_status sweep_impl(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *qhost, const float *qdev, int k,
                            int batch, float *peak, int *argmax, int out_on_device, Weights w = Weights())
{
    if (batch == 0) batch = c->sweep_batch;
    const int N = c->g.N, H = c->g.H;
    cudaStream_t st = c->stream;
    cudaError_t e;
    const size_t key_bytes = sizeof(unsigned long long) * (size_t)k;
    const size_t out_bytes = out_on_device ? 0 : (sizeof(float) + sizeof(int)) * (size_t)k;
    if ((e = c->ws.keys.ensure(key_bytes + out_bytes, false, st)) != cudaSuccess) return cuda_fail(e, "keys");
    unsigned long long *keys = (unsigned long long *)c->ws.keys.p;
    if ((e = cudaMemsetAsync(keys, 0, key_bytes, st)) != cudaSuccess) return cuda_fail(e, "clear keys");
    {
        std::vector<bc_shape_t> shapes(1, A);
        std::vector<const float *> q(1, nullptr);
        std::vector<PairDesc> pairs(1, PairDesc{0, -1, 0, 0, 0});
        if (bc_status s = enqueue(c, shapes, q, pairs, true, nullptr, nullptr, nullptr, w)) return s;
    }
    for (int r0 = 0; r0 < k; r0 += batch) {
        const int nb = std::min(batch, k - r0);
        std::vector<bc_shape_t> shapes(nb, B);
        std::vector<const float *> q(nb, nullptr), qd(nb, nullptr);
        std::vector<PairDesc> pairs(nb);
        for (int i = 0; i < nb; i++) {
            if (qhost) q[i] = qhost + 4 * (size_t)(r0 + i);
            else qd[i] = qdev + 4 * (size_t)(r0 + i);
            pairs[i] = PairDesc{-1, i, (long long)i * N * N * H, 0, (long long)(r0 + i)};
        }
        if (bc_status s = enqueue(c, shapes, q, pairs, false, nullptr, keys, qhost ? nullptr : &qd, w)) return s;
    }
    float *dpeak = peak;
    int *darg = argmax;
    if (!out_on_device) {
        dpeak = (float *)((char *)c->ws.keys.p + key_bytes);
        darg = (int *)(dpeak + k);
    }
    if ((e = launch_decode_peaks(keys, k, dpeak, darg, st)) != cudaSuccess) return cuda_fail(e, "decode peaks");
    if (!out_on_device) {
        if ((e = cudaMemcpyAsync(peak, dpeak, sizeof(float) * (size_t)k, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "copy peaks");
        if ((e = cudaMemcpyAsync(argmax, darg, sizeof(int) * (size_t)k, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(e, "copy argmax");
        return bc_sync(c);
    }
    return BC_OK;
}

// A host-resident result in mapped page-locked memory is stored by the kernels
// directly; any other host memory goes through a device staging buffer and one
// copy.
static float *mapped_host(float *p) { return (float *)mapped_host_ptr(p); }

static bc_status check_quats(const float *quats, int k, const char *who)
{
    for (int r = 0; r < k; r++) {
        const float *q = quats + 4 * r;
        const double n2 = (double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3];
        if (!(n2 > 1e-30) || !std::isfinite(n2)) return fail(BC_ERR_ARG, std::string(who) + ": zero or non-finite quaternion");
    }
    return BC_OK;
}

extern "C" {

static bc_status correlate_impl(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, float *out,
                                int out_on_device, Weights w, const char *who)
{
    try {
        if (!c || !A || !B || !quats || !out) return fail(BC_ERR_ARG, std::string(who) + ": null argument");
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, std::string(who) + ": shapes belong to another context");
        if (k < 1 || k > 65534) return fail(BC_ERR_ARG, std::string(who) + ": k must be in [1, 65534]");
        if (bc_status s = check_quats(quats, k, who)) return s;
        const int N = c->g.N, H = c->g.H;
        const long long N3 = (long long)N * N * N;
        std::vector<bc_shape_t> shapes(1 + k, B);
        shapes[0] = A;
        std::vector<const float *> q(1 + k, nullptr);
        for (int r = 0; r < k; r++) q[1 + r] = quats + 4 * r;
        const bool fused = (k == 1);
        std::vector<PairDesc> pairs;
        if (!fused) pairs.push_back(PairDesc{0, -1, 0, 0, 0}); // spectrum of A into the cache
        for (int r = 0; r < k; r++)
            pairs.push_back(PairDesc{fused ? 0 : -1, 1 + r, (long long)r * N * N * H, (long long)r * N3, r});
        float *dout = out;
        float *mapped = out_on_device ? nullptr : mapped_host(out);
        cudaError_t e;
        if (mapped) {
            dout = mapped;
        } else if (!out_on_device) {
            if ((e = c->outbuf.ensure(sizeof(float) * (size_t)k * N3, false, c->stream)) != cudaSuccess) return cuda_fail(e, "outbuf");
            dout = (float *)c->outbuf.p;
        }
        if (bc_status s = enqueue(c, shapes, q, pairs, !fused, dout, nullptr, nullptr, w)) return s;
        if (!out_on_device) {
            if (!mapped &&
                (e = cudaMemcpyAsync(out, dout, sizeof(float) * (size_t)k * N3, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
                return cuda_fail(e, "copy out");
            return bc_sync(c);
        }
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, std::string(who) + ": unexpected exception");
    }
}

bc_status bc_correlate(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, float *out,
                       int out_on_device)
{
    return correlate_impl(c, A, B, quats, k, out, out_on_device, Weights(), "bc_correlate");
}

// The complementarity weights for (r0, lambda), rebuilt on the context stream
// when the parameters change (stream order keeps earlier calls on the old ones).
static bc_status score_weights(bc_ctx_t c, double r0, double lambda, const char *who, Weights *w)
{
    if (!(r0 >= 0) || !std::isfinite(r0) || !(lambda >= 0) || !std::isfinite(lambda))
        return fail(BC_ERR_ARG, std::string(who) + ": r0 and lambda must be finite and >= 0");
    const size_t n = (size_t)c->g.L * (c->qmax + 1);
    cudaError_t e;
    const size_t before = c->score_ft.bytes;
    if ((e = c->score_ft.ensure(sizeof(float) * n, false, c->stream)) != cudaSuccess) return cuda_fail(e, who);
    if ((e = c->score_xw.ensure(sizeof(float) * xw_floats(c->g), false, c->stream)) != cudaSuccess) return cuda_fail(e, who);
    if (c->score_ft.bytes != before || r0 != c->score_r0 || lambda != c->score_lambda) {
        if ((e = launch_build_score_table(c->g, c->period, c->radii_dev, r0, lambda, (float *)c->score_ft.p, c->stream)) != cudaSuccess)
            return cuda_fail(e, who);
        if ((e = launch_build_xw(c->g, c->deconv, (const float *)c->score_ft.p, (float *)c->score_xw.p, c->stream)) != cudaSuccess)
            return cuda_fail(e, who);
        c->score_r0 = r0;
        c->score_lambda = lambda;
    }
    w->ballft = (const float *)c->score_ft.p;
    w->xw = (const float *)c->score_xw.p;
    w->sign = -1.f;
    return BC_OK;
}

bc_status bc_score(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, double r0, double lambda,
                   float *out, int out_on_device)
{
    try {
        if (!c) return fail(BC_ERR_ARG, "bc_score: null context");
        Weights w;
        if (bc_status s = score_weights(c, r0, lambda, "bc_score", &w)) return s;
        return correlate_impl(c, A, B, quats, k, out, out_on_device, w, "bc_score");
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_score: unexpected exception");
    }
}

bc_status bc_pairs(bc_ctx_t c, const bc_shape_t *As, const bc_shape_t *Bs, const float *quats, int npairs,
                   float *out, float *peak, int *argmax, int on_device)
{
    try {
        if (!c || !As || !Bs || !quats) return fail(BC_ERR_ARG, "bc_pairs: null argument");
        if (!out && !peak) return fail(BC_ERR_ARG, "bc_pairs: nothing to compute (out and peak are null)");
        if ((peak == nullptr) != (argmax == nullptr)) return fail(BC_ERR_ARG, "bc_pairs: peak and argmax go together");
        if (npairs < 1 || npairs > 32767) return fail(BC_ERR_ARG, "bc_pairs: npairs must be in [1, 32767]");
        for (int i = 0; i < npairs; i++) {
            if (!As[i] || !Bs[i]) return fail(BC_ERR_ARG, "bc_pairs: null shape");
            if (As[i]->ctx != c || Bs[i]->ctx != c) return fail(BC_ERR_ARG, "bc_pairs: shapes belong to another context");
        }
        if (bc_status s = check_quats(quats, npairs, "bc_pairs")) return s;
        const int N = c->g.N, H = c->g.H;
        const long long N3 = (long long)N * N * N;
        cudaStream_t st = c->stream;
        cudaError_t e;
        const size_t key_bytes = peak ? sizeof(unsigned long long) * (size_t)npairs : 0;
        const size_t pk_bytes = (peak && !on_device) ? (sizeof(float) + sizeof(int)) * (size_t)npairs : 0;
        if (key_bytes && (e = c->ws.keys.ensure(key_bytes + pk_bytes, false, st)) != cudaSuccess) return cuda_fail(e, "keys");
        unsigned long long *keys = key_bytes ? (unsigned long long *)c->ws.keys.p : nullptr;
        if (keys && (e = cudaMemsetAsync(keys, 0, key_bytes, st)) != cudaSuccess) return cuda_fail(e, "clear keys");
        float *dout = out;
        float *mapped = (out && !on_device) ? mapped_host(out) : nullptr;
        if (mapped) {
            dout = mapped;
        } else if (out && !on_device) {
            if ((e = c->outbuf.ensure(sizeof(float) * (size_t)npairs * N3, false, st)) != cudaSuccess) return cuda_fail(e, "outbuf");
            dout = (float *)c->outbuf.p;
        }
        std::vector<bc_shape_t> shapes(2 * (size_t)npairs);
        std::vector<const float *> q(2 * (size_t)npairs, nullptr);
        std::vector<PairDesc> pairs(npairs);
        for (int i = 0; i < npairs; i++) {
            shapes[2 * i] = As[i];
            shapes[2 * i + 1] = Bs[i];
            q[2 * i + 1] = quats + 4 * (size_t)i;
            pairs[i] = PairDesc{2 * i, 2 * i + 1, (long long)i * N * N * H, (long long)i * N3, i};
        }
        if (bc_status s = enqueue(c, shapes, q, pairs, false, dout, keys)) return s;
        if (peak) {
            float *dpeak = peak;
            int *darg = argmax;
            if (!on_device) {
                dpeak = (float *)((char *)c->ws.keys.p + key_bytes);
                darg = (int *)(dpeak + npairs);
            }
            if ((e = launch_decode_peaks(keys, npairs, dpeak, darg, st)) != cudaSuccess) return cuda_fail(e, "decode peaks");
            if (!on_device) {
                if ((e = cudaMemcpyAsync(peak, dpeak, sizeof(float) * npairs, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                    return cuda_fail(e, "copy peaks");
                if ((e = cudaMemcpyAsync(argmax, darg, sizeof(int) * npairs, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                    return cuda_fail(e, "copy argmax");
            }
        }
        if (out && !on_device && !mapped) {
            if ((e = cudaMemcpyAsync(out, dout, sizeof(float) * (size_t)npairs * N3, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_fail(e, "copy out");
        }
        if (!on_device) return bc_sync(c);
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_pairs: unexpected exception");
    }
}

bc_status bc_sweep(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, float *peak,
                   int *argmax, int out_on_device)
{
    try {
        if (!c || !A || !B || !quats || !peak || !argmax) return fail(BC_ERR_ARG, "bc_sweep: null argument");
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_sweep: shapes belong to another context");
        if (k < 1 || k > (1 << 24)) return fail(BC_ERR_ARG, "bc_sweep: k must be in [1, 2^24]");
        if (batch < 0 || batch > 65534) return fail(BC_ERR_ARG, "bc_sweep: batch must be in [0, 65534]");
        if (bc_status s = check_quats(quats, k, "bc_sweep")) return s;
        return sweep_impl(c, A, B, quats, nullptr, k, batch, peak, argmax, out_on_device);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_sweep: unexpected exception");
    }
}

bc_status bc_score_sweep(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, double r0,
                         double lambda, float *peak, int *argmax, int out_on_device)
{
    try {
        if (!c || !A || !B || !quats || !peak || !argmax) return fail(BC_ERR_ARG, "bc_score_sweep: null argument");
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_score_sweep: shapes belong to another context");
        if (k < 1 || k > (1 << 24)) return fail(BC_ERR_ARG, "bc_score_sweep: k must be in [1, 2^24]");
        if (batch < 0 || batch > 65534) return fail(BC_ERR_ARG, "bc_score_sweep: batch must be in [0, 65534]");
        if (bc_status s = check_quats(quats, k, "bc_score_sweep")) return s;
        Weights w;
        if (bc_status s = score_weights(c, r0, lambda, "bc_score_sweep", &w)) return s;
        return sweep_impl(c, A, B, quats, nullptr, k, batch, peak, argmax, out_on_device, w);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_score_sweep: unexpected exception");
    }
}

bc_status bc_sweep_plan(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, float *peak,
                        int *argmax, bc_plan_t *out)
{
    bc_plan_s *pl = nullptr;
    try {
        if (!c || !A || !B || !quats || !peak || !argmax || !out) return fail(BC_ERR_ARG, "bc_sweep_plan: null argument");
        *out = nullptr;
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_sweep_plan: shapes belong to another context");
        if (k < 1 || k > (1 << 24)) return fail(BC_ERR_ARG, "bc_sweep_plan: k must be in [1, 2^24]");
        if (batch < 0 || batch > 65534) return fail(BC_ERR_ARG, "bc_sweep_plan: batch must be in [0, 65534]");
        if (bc_status s = check_quats(quats, k, "bc_sweep_plan")) return s;
        if (batch == 0) batch = c->sweep_batch;
        const int N = c->g.N, H = c->g.H;
        cudaStream_t st = c->stream;
        cudaError_t e;
        pl = new bc_plan_s();
        pl->ctx = c;
        pl->k = k;
        // plan every pass on the host
        std::vector<Job> jobs;
        jobs.push_back(plan_job(c, std::vector<bc_shape_t>(1, A), std::vector<const float *>(1, nullptr),
                                std::vector<PairDesc>(1, PairDesc{0, -1, 0, 0, 0}), true, nullptr));
        for (int r0 = 0; r0 < k; r0 += batch) {
            const int nb = std::min(batch, k - r0);
            std::vector<const float *> q(nb);
            std::vector<PairDesc> pairs(nb);
            for (int i = 0; i < nb; i++) {
                q[i] = quats + 4 * (size_t)(r0 + i);
                pairs[i] = PairDesc{-1, i, (long long)i * N * N * H, 0, (long long)(r0 + i)};
            }
            jobs.push_back(plan_job(c, std::vector<bc_shape_t>(nb, B), q, pairs, false, nullptr));
        }
        long long mk = 0, mi = 0, mp = 0, mg = 0, mz = 0, my = 0, mh = 0;
        std::vector<size_t> doff(jobs.size());
        size_t dbytes = 0;
        for (size_t j = 0; j < jobs.size(); j++) {
            const Job &jb = jobs[j];
            mk = std::max(mk, (long long)jb.koff);
            mi = std::max(mi, (long long)jb.inst.size());
            mp = std::max(mp, (long long)jb.pairs.size());
            mg = std::max(mg, jb.goff);
            mz = std::max(mz, jb.zoff);
            my = std::max(my, jb.yoff);
            mh = std::max(mh, jb.hpairs);
            doff[j] = dbytes;
            dbytes += (sizeof(InstDesc) * jb.inst.size() + sizeof(PairDesc) * jb.pairs.size() + 255) & ~size_t(255);
        }
        if (bc_status s = ensure_ws(c, pl->ws, jobs[0].mode, mk, mi, mp, mg, mz, my, mh)) {
            bc_plan_destroy(pl);
            return s;
        }
        if ((e = pl->ws.keys.ensure(sizeof(unsigned long long) * (size_t)k, false, st)) != cudaSuccess ||
            (e = pl->desc.ensure(dbytes, false, st)) != cudaSuccess) {
            bc_plan_destroy(pl);
            return cuda_fail(e, "bc_sweep_plan: workspace");
        }
        std::vector<char> host(dbytes);
        for (size_t j = 0; j < jobs.size(); j++) {
            const size_t ib = sizeof(InstDesc) * jobs[j].inst.size();
            std::memcpy(host.data() + doff[j], jobs[j].inst.data(), ib);
            std::memcpy(host.data() + doff[j] + ib, jobs[j].pairs.data(), sizeof(PairDesc) * jobs[j].pairs.size());
        }
        if ((e = cudaMemcpyAsync(pl->desc.p, host.data(), dbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            bc_plan_destroy(pl);
            return cuda_fail(e, "bc_sweep_plan: descriptors");
        }
        // capture: clear keys, A's spectrum, every batch, decode -- on a private stream (the
        // legacy default stream cannot be captured); the graph later runs on ctx's stream
        unsigned long long *keys = (unsigned long long *)pl->ws.keys.p;
        cudaStream_t cs = nullptr;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
            bc_plan_destroy(pl);
            return cuda_fail(e, "bc_sweep_plan: capture stream");
        }
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
            cudaStreamDestroy(cs);
            bc_plan_destroy(pl);
            return cuda_fail(e, "bc_sweep_plan: begin capture");
        }
        bc_status s = BC_OK;
        if ((e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)k, cs)) != cudaSuccess)
            s = cuda_fail(e, "bc_sweep_plan: clear keys");
        for (size_t j = 0; s == BC_OK && j < jobs.size(); j++) {
            const char *base = (const char *)pl->desc.p + doff[j];
            s = launch_job(c, pl->ws, jobs[j], (const InstDesc *)base,
                           (const PairDesc *)(base + sizeof(InstDesc) * jobs[j].inst.size()), nullptr,
                           j == 0 ? nullptr : keys, false, cs, &pl->launches);
        }
        if (s == BC_OK && (e = launch_decode_peaks(keys, k, peak, argmax, cs)) != cudaSuccess)
            s = cuda_fail(e, "bc_sweep_plan: decode");
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (s == BC_OK && e != cudaSuccess) s = cuda_fail(e, "bc_sweep_plan: end capture");
        if (s == BC_OK && (e = cudaGraphInstantiate(&pl->exec, graph, 0)) != cudaSuccess)
            s = cuda_fail(e, "bc_sweep_plan: instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (s != BC_OK) {
            bc_plan_destroy(pl);
            return s;
        }
        pl->launches += 1; // the peak decode
        *out = pl;
        return BC_OK;
    } catch (...) {
        if (pl) bc_plan_destroy(pl);
        return fail(BC_ERR_INTERNAL, "bc_sweep_plan: unexpected exception");
    }
}

bc_status bc_plan_run(bc_plan_t pl)
{
    if (!pl || !pl->exec) return fail(BC_ERR_ARG, "bc_plan_run: null or empty plan");
    CK(cudaGraphLaunch(pl->exec, pl->ctx->stream));
    return BC_OK;
}

bc_status bc_plan_destroy(bc_plan_t pl)
{
    if (!pl) return BC_OK;
    if (pl->ctx) cudaStreamSynchronize(pl->ctx->stream);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    pl->ws.release();
    pl->desc.release();
    delete pl;
    return BC_OK;
}

// Moments of S rotated by the host quaternion rot (null: not rotated): the
// shape's spectrum through the correlation pipeline, then the mode magnitudes.
static bc_status shape_moments(bc_ctx_t c, bc_shape_t S, const float *rot, float *out)
{
    std::vector<bc_shape_t> shapes(1, S);
    std::vector<const float *> q(1, rot);
    std::vector<PairDesc> pairs(1, PairDesc{0, -1, 0, 0, 0});
    if (bc_status s = enqueue(c, shapes, q, pairs, true, nullptr, nullptr)) return s;
    cudaError_t e = launch_moments((const float2 *)c->ws.fa.p, c->modes, BC_MOMENTS, c->g.N, c->g.H, out, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments");
    return BC_OK;
}

bc_status bc_shape_moments(bc_ctx_t c, bc_shape_t S, float *out)
{
    try {
        if (!c || !S || !out) return fail(BC_ERR_ARG, "bc_shape_moments: null argument");
        if (S->ctx != c) return fail(BC_ERR_ARG, "bc_shape_moments: shape belongs to another context");
        if (S->n == 0) return fail(BC_ERR_ARG, "bc_shape_moments: empty shape (f(0) = 0)");
        return shape_moments(c, S, nullptr, out);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_shape_moments: unexpected exception");
    }
}

bc_status bc_shape_moments_rot(bc_ctx_t c, bc_shape_t S, const float *quats, int n, float *out)
{
    try {
        if (!c || !S || !quats || !out) return fail(BC_ERR_ARG, "bc_shape_moments_rot: null argument");
        if (S->ctx != c) return fail(BC_ERR_ARG, "bc_shape_moments_rot: shape belongs to another context");
        if (S->n == 0) return fail(BC_ERR_ARG, "bc_shape_moments_rot: empty shape (f(0) = 0)");
        if (n < 1) return fail(BC_ERR_ARG, "bc_shape_moments_rot: n < 1");
        cudaError_t e = launch_moments_rot(S->knots, S->n, quats, n, c->ballft, c->qmax + 1, c->g.L,
                                           (float)(2.0 / c->period), out, c->err_dev, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "moments of rotated shapes");
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_shape_moments_rot: unexpected exception");
    }
}

bc_status bc_topk(bc_ctx_t c, const float *scores, int n, int k, int *idx)
{
    if (!c || !scores || !idx) return fail(BC_ERR_ARG, "bc_topk: null argument");
    if (n < 1 || n > BC_TOPK_MAX || k < 1 || k > n) return fail(BC_ERR_ARG, "bc_topk: need 1 <= k <= n <= 16384");
    cudaError_t e = launch_topk(scores, n, k, idx, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "top-k");
    return BC_OK;
}

bc_status bc_learned_sweep_avg(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                               int topk, const float *orients, int norient, int *idx, float *peak, int *argmax,
                               float *scores)
{
    try {
        if (!c || !net || !A || !B || !quats || !idx || !peak || !argmax)
            return fail(BC_ERR_ARG, "bc_learned_sweep: null argument");
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_learned_sweep: shapes belong to another context");
        if (n < 1 || n > BC_TOPK_MAX) return fail(BC_ERR_ARG, "bc_learned_sweep: n must be in [1, 16384]");
        if (topk < 1 || topk > n) return fail(BC_ERR_ARG, "bc_learned_sweep: topk must be in [1, n]");
        if (norient < 0 || (norient > 0 && !orients))
            return fail(BC_ERR_ARG, "bc_learned_sweep: norient < 0, or orientations missing");
        if (A->n == 0 || B->n == 0) return fail(BC_ERR_ARG, "bc_learned_sweep: empty shape (f(0) = 0)");
        if (norient > 0)
            if (bc_status s = check_quats(orients, norient, "bc_learned_sweep")) return s;
        cudaStream_t st = c->stream;
        cudaError_t e;
        const bool rot = bc_mlp_rotated_moments(net) != 0;
        // scratch: moments (2 x 64), features (n x 144), scores (n), score sum (n),
        // composed rotations (n x 4), selected rotations (topk x 4), and the rotated
        // ligand's moments (n x 64) when the network takes those
        const size_t fbytes = sizeof(float) * (2 * BC_MOMENTS + (size_t)n * 144 + 2 * (size_t)n + 4 * (size_t)n +
                                               4 * (size_t)topk + (rot ? (size_t)n * BC_MOMENTS : 0));
        if ((e = c->learn.ensure(fbytes, false, st)) != cudaSuccess) return cuda_fail(e, "learned scratch");
        float *fa = (float *)c->learn.p, *fb = fa + BC_MOMENTS, *X = fb + BC_MOMENTS;
        float *sc = X + (size_t)n * 144, *acc = sc + n, *qs = acc + n, *qsel = qs + 4 * (size_t)n;
        float *fbr = qsel + 4 * (size_t)topk;
        float *total = scores ? scores : acc;
        // features of rotations `q` against the receptor moments in fa
        auto features = [&](const float *q) -> bc_status {
            if (!rot) return bc_mlp_features(net, q, n, fa, fb, X);
            cudaError_t e2 = launch_moments_rot(B->knots, B->n, q, n, c->ballft, c->qmax + 1, c->g.L,
                                                (float)(2.0 / c->period), fbr, c->err_dev, st);
            if (e2 != cudaSuccess) return cuda_fail(e2, "moments of the rotated ligand");
            return bc_mlp_features_rows(net, q, n, fa, fbr, X);
        };
        if (bc_status s = shape_moments(c, A, nullptr, fa)) return s;
        if (!rot)
            if (bc_status s = shape_moments(c, B, nullptr, fb)) return s;
        if (bc_status s = features(quats)) return s;
        if (bc_status s = bc_mlp_predict(net, X, n, total)) return s;
        // (S A, S R B) has the same peak over translations as (A, R B): score the
        // rotations S R of B against the receptor turned by S, and average
        for (int k = 0; k < norient; k++) {
            const float *s4 = orients + 4 * (size_t)k;
            if (bc_status s = shape_moments(c, A, s4, fa)) return s;
            if ((e = launch_compose_quats(s4, quats, n, qs, st)) != cudaSuccess) return cuda_fail(e, "compose rotations");
            if (bc_status s = features(qs)) return s;
            if (bc_status s = bc_mlp_predict(net, X, n, sc)) return s;
            if ((e = launch_axpby(total, sc, n, 1.f, 1.f, st)) != cudaSuccess) return cuda_fail(e, "score sum");
        }
        if (norient > 0 && (e = launch_axpby(total, total, n, 1.f / (float)(norient + 1), 0.f, st)) != cudaSuccess)
            return cuda_fail(e, "score mean");
        if ((e = launch_topk(total, n, topk, idx, st)) != cudaSuccess) return cuda_fail(e, "top-k");
        if ((e = launch_gather_quats(quats, idx, topk, qsel, st)) != cudaSuccess) return cuda_fail(e, "gather rotations");
        return sweep_impl(c, A, B, nullptr, qsel, topk, 0, peak, argmax, 1);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_learned_sweep: unexpected exception");
    }
}

bc_status bc_learned_sweep(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n, int topk,
                           int *idx, float *peak, int *argmax, float *scores)
{
    return bc_learned_sweep_avg(c, net, A, B, quats, n, topk, nullptr, 0, idx, peak, argmax, scores);
}

// ------------------------------------------------------------------ learned sweep, two stages
namespace {
__global__ void k_gather_scores(const float *__restrict__ x, const int *__restrict__ idx, int k, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = x[idx[i]];
}
__global__ void k_compose_idx(const int *__restrict__ outer, const int *__restrict__ inner, int k, int *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = outer[inner[i]];
}
} // namespace

// The network's ranking of the two-stage learned sweeps: stage 1 scores all n
// rotations with one view and keeps the best `keep`; stage 2 scores those again
// against the receptor turned by each orientation and ranks them by the mean of
// the views; the best m are written to idx_out (indices into quats, device, m
// ints) and their rotations to *q_out (device, 4 m floats, inside the learned
// scratch); with idx_out null the indices go to the scratch as well, at
// *picks.  `extra` bytes of the scratch, after the ranking's own, are handed to
// the caller at *extra_out (256-byte aligned).  The caller validates.
static bc_status learned_rank(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n, int m,
                              const float *orients, int norient, int keep, float *scores, int *idx_out,
                              const int **picks, const float **q_out, size_t extra, void **extra_out)
{
    cudaStream_t st = c->stream;
    cudaError_t e;
    const bool rot = bc_mlp_rotated_moments(net) != 0;
    const size_t M = BC_MOMENTS, no = (size_t)norient, kp = (size_t)keep, N = (size_t)n;
    // scratch (floats): receptor and ligand moments (2 M), features (n x 144), one-view
    // scores (n), kept sums and scores (2 keep), kept and composed rotations (2 x 4 keep),
    // selected rotations (4 m), turned-receptor moments (norient M) and orientations
    // (4 norient), rotated-ligand moments (n M, when the network takes them); ints: kept
    // and selected indices and the picks (keep + 2 m); then the caller's extra bytes
    const size_t nf = 2 * M + N * 144 + N + 2 * kp + 8 * kp + 4 * (size_t)m + no * M + 4 * no + (rot ? N * M : 0);
    const size_t own = ((sizeof(float) * nf + sizeof(int) * (kp + 2 * (size_t)m)) + 255) & ~(size_t)255;
    if ((e = c->learn.ensure(own + extra, false, st)) != cudaSuccess) return cuda_fail(e, "learned scratch");
    float *fa = (float *)c->learn.p, *fb = fa + M, *X = fb + M, *s0 = X + N * 144, *acc = s0 + N, *sc = acc + kp;
    float *q1 = sc + kp, *qs = q1 + 4 * kp, *qsel = qs + 4 * kp, *fo = qsel + 4 * (size_t)m, *od = fo + no * M;
    float *fbr = od + 4 * no;
    int *i1 = (int *)(fbr + (rot ? N * M : 0)), *i2 = i1 + kp, *ip = i2 + m;
    if (!idx_out) idx_out = ip;
    if (picks) *picks = idx_out;
    if (extra_out) *extra_out = (char *)c->learn.p + own;
    auto features = [&](const float *q, int rows, const float *fA) -> bc_status {
        if (!rot) return bc_mlp_features(net, q, rows, fA, fb, X);
        cudaError_t e2 = launch_moments_rot(B->knots, B->n, q, rows, c->ballft, c->qmax + 1, c->g.L,
                                            (float)(2.0 / c->period), fbr, c->err_dev, st);
        if (e2 != cudaSuccess) return cuda_fail(e2, "moments of the rotated ligand");
        return bc_mlp_features_rows(net, q, rows, fA, fbr, X);
    };
    float *s_all = scores ? scores : s0;
    // stage 1: one view for every rotation, keep the best `keep`
    if (bc_status s = shape_moments(c, A, nullptr, fa)) return s;
    if (!rot)
        if (bc_status s = shape_moments(c, B, nullptr, fb)) return s;
    if (bc_status s = features(quats, n, fa)) return s;
    if (bc_status s = bc_mlp_predict(net, X, n, s_all)) return s;
    if ((e = launch_topk(s_all, n, keep, i1, st)) != cudaSuccess) return cuda_fail(e, "top-k (kept)");
    if ((e = launch_gather_quats(quats, i1, keep, q1, st)) != cudaSuccess) return cuda_fail(e, "gather kept rotations");
    k_gather_scores<<<(keep + 255) / 256, 256, 0, st>>>(s_all, i1, keep, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gather kept scores");
    // stage 2: the kept rotations against the receptor turned by each orientation S_k,
    // whose moments come from one direct-sum launch over all orientations
    if (norient > 0) {
        if ((e = cudaMemcpyAsync(od, orients, sizeof(float) * 4 * no, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "orientations");
        if ((e = launch_moments_rot(A->knots, A->n, od, norient, c->ballft, c->qmax + 1, c->g.L,
                                    (float)(2.0 / c->period), fo, c->err_dev, st)) != cudaSuccess)
            return cuda_fail(e, "moments of the turned receptor");
    }
    for (int k = 0; k < norient; k++) {
        if ((e = launch_compose_quats(orients + 4 * (size_t)k, q1, keep, qs, st)) != cudaSuccess)
            return cuda_fail(e, "compose rotations");
        if (bc_status s = features(qs, keep, fo + (size_t)k * M)) return s;
        if (bc_status s = bc_mlp_predict(net, X, keep, sc)) return s;
        if ((e = launch_axpby(acc, sc, keep, 1.f, 1.f, st)) != cudaSuccess) return cuda_fail(e, "score sum");
    }
    if (norient > 0 && (e = launch_axpby(acc, acc, keep, 1.f / (float)(norient + 1), 0.f, st)) != cudaSuccess)
        return cuda_fail(e, "score mean");
    if ((e = launch_topk(acc, keep, m, i2, st)) != cudaSuccess) return cuda_fail(e, "top-k");
    k_compose_idx<<<(m + 255) / 256, 256, 0, st>>>(i1, i2, m, idx_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "rotation indices");
    if ((e = launch_gather_quats(q1, i2, m, qsel, st)) != cudaSuccess) return cuda_fail(e, "gather rotations");
    *q_out = qsel;
    return BC_OK;
}

// Arguments shared by the two-stage learned sweeps.
static bc_status check_learned(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                               int topk, const float *orients, int norient, int keep, int *idx, float *peak,
                               int *argmax, const char *who)
{
    if (!c || !net || !A || !B || !quats || !idx || !peak || !argmax) return fail(BC_ERR_ARG, std::string(who) + ": null argument");
    if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, std::string(who) + ": shapes belong to another context");
    if (n < 1 || n > BC_TOPK_MAX) return fail(BC_ERR_ARG, std::string(who) + ": n must be in [1, 16384]");
    if (keep < 1 || keep > n) return fail(BC_ERR_ARG, std::string(who) + ": keep must be in [1, n]");
    if (topk < 1 || topk > keep) return fail(BC_ERR_ARG, std::string(who) + ": topk must be in [1, keep]");
    if (norient < 0 || (norient > 0 && !orients))
        return fail(BC_ERR_ARG, std::string(who) + ": norient < 0, or orientations missing");
    if (A->n == 0 || B->n == 0) return fail(BC_ERR_ARG, std::string(who) + ": empty shape (f(0) = 0)");
    if (norient > 0)
        if (bc_status s = check_quats(orients, norient, who)) return s;
    return BC_OK;
}

bc_status bc_learned_sweep_cascade(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                                   int topk, const float *orients, int norient, int keep, int *idx, float *peak,
                                   int *argmax, float *scores)
{
    try {
        if (bc_status s = check_learned(c, net, A, B, quats, n, topk, orients, norient, keep, idx, peak, argmax,
                                        "bc_learned_sweep_cascade"))
            return s;
        const float *qsel = nullptr;
        if (bc_status s = learned_rank(c, net, A, B, quats, n, topk, orients, norient, keep, scores, idx, nullptr,
                                       &qsel, 0, nullptr))
            return s;
        return sweep_impl(c, A, B, nullptr, qsel, topk, 0, peak, argmax, 1);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_learned_sweep_cascade: unexpected exception");
    }
}

bc_status bc_learned_sweep_coarse(bc_ctx_t c, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                                  int topk, const float *orients, int norient, int keep, bc_ctx_t cc, bc_shape_t Ac,
                                  bc_shape_t Bc, int coarse_keep, int *idx, float *peak, int *argmax, float *scores)
{
    try {
        const char *who = "bc_learned_sweep_coarse";
        if (bc_status s = check_learned(c, net, A, B, quats, n, coarse_keep, orients, norient, keep, idx, peak,
                                        argmax, who))
            return s;
        if (!cc || !Ac || !Bc) return fail(BC_ERR_ARG, "bc_learned_sweep_coarse: null coarse context or shape");
        if (Ac->ctx != cc || Bc->ctx != cc)
            return fail(BC_ERR_ARG, "bc_learned_sweep_coarse: coarse shapes belong to another context");
        if (topk < 1 || topk > coarse_keep) return fail(BC_ERR_ARG, "bc_learned_sweep_coarse: topk must be in [1, coarse_keep]");
        if (Ac->n != A->n || Bc->n != B->n)
            return fail(BC_ERR_ARG, "bc_learned_sweep_coarse: coarse shapes have other knot counts than A and B");
        if (cc->radii != c->radii || cc->period != c->period)
            return fail(BC_ERR_ARG, "bc_learned_sweep_coarse: the coarse context has other radius levels or another period");
        cudaStream_t st = c->stream;
        cudaError_t e;
        const size_t cm = (size_t)coarse_keep, tk = (size_t)topk;
        // extra scratch: coarse peaks (cm floats), selected rotations (4 topk floats), coarse
        // argmax (cm ints), the coarse ranking (topk ints)
        const size_t extra = sizeof(float) * (cm + 4 * tk) + sizeof(int) * (cm + tk);
        void *ex = nullptr;
        const int *picks = nullptr;
        const float *qm = nullptr;
        // stages 1-2: the network's best coarse_keep
        if (bc_status s = learned_rank(c, net, A, B, quats, n, coarse_keep, orients, norient, keep, scores, nullptr,
                                       &picks, &qm, extra, &ex))
            return s;
        float *cpeak = (float *)ex, *qsel = cpeak + cm;
        int *carg = (int *)(qsel + 4 * tk), *i3 = carg + cm;
        // stage 3: their correlations at the coarse band limit, on the coarse context's stream
        const bool two = cc->stream != st;
        if (two) {
            if (!c->ev_a && (e = cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "event");
            if (!c->ev_b && (e = cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "event");
            if ((e = cudaEventRecord(c->ev_a, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cc->stream, c->ev_a, 0)) != cudaSuccess)
                return cuda_fail(e, "order the coarse stage after the ranking");
        }
        if (bc_status s = sweep_impl(cc, Ac, Bc, nullptr, qm, coarse_keep, 0, cpeak, carg, 1)) return s;
        if (two) {
            if ((e = cudaEventRecord(c->ev_b, cc->stream)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c->ev_b, 0)) != cudaSuccess)
                return cuda_fail(e, "order the full stage after the coarse one");
        }
        // stage 4: the best topk by their coarse peaks get full correlations
        if ((e = launch_topk(cpeak, coarse_keep, topk, i3, st)) != cudaSuccess) return cuda_fail(e, "top-k (coarse)");
        k_compose_idx<<<(topk + 255) / 256, 256, 0, st>>>(picks, i3, topk, idx);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "rotation indices");
        if ((e = launch_gather_quats(qm, i3, topk, qsel, st)) != cudaSuccess) return cuda_fail(e, "gather rotations");
        return sweep_impl(c, A, B, nullptr, qsel, topk, 0, peak, argmax, 1);
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_learned_sweep_coarse: unexpected exception");
    }
}

// ------------------------------------------------------------------ tuning

bc_status bc_get_tuning(bc_ctx_t c, bc_tuning *out)
{
    if (!c || !out) return fail(BC_ERR_ARG, "bc_get_tuning: null argument");
    out->spread = c->spread_mode;
    out->sweep_batch = c->sweep_batch;
    out->graphs = c->replay ? 1 : 0;
    out->fft_schedule = c->fft_sched;
    out->z_transform = c->z_tc;
    out->persistent = c->persistent;
    out->overlap = c->overlap;
    return BC_OK;
}

bc_status bc_set_tuning(bc_ctx_t c, const bc_tuning *t)
{
    if (!c || !t) return fail(BC_ERR_ARG, "bc_set_tuning: null argument");
    if (t->spread != 0 && t->spread != 1) return fail(BC_ERR_ARG, "bc_set_tuning: spread must be 0 or 1");
    if (t->sweep_batch < 1 || t->sweep_batch > 65534) return fail(BC_ERR_ARG, "bc_set_tuning: sweep_batch must be in [1, 65534]");
    if (t->graphs != 0 && t->graphs != 1) return fail(BC_ERR_ARG, "bc_set_tuning: graphs must be 0 or 1");
    if (t->fft_schedule < 0 || t->fft_schedule > 7) return fail(BC_ERR_ARG, "bc_set_tuning: fft_schedule must be in [0, 7]");
    if (t->z_transform != 0 && t->z_transform != 1) return fail(BC_ERR_ARG, "bc_set_tuning: z_transform must be 0 or 1");
    if (t->persistent != 0 && t->persistent != 1) return fail(BC_ERR_ARG, "bc_set_tuning: persistent must be 0 or 1");
    if (t->overlap != 0 && t->overlap != 1) return fail(BC_ERR_ARG, "bc_set_tuning: overlap must be 0 or 1");
    if (t->z_transform == 1 && !c->zdft)
        return fail(BC_ERR_UNSUPPORTED, "bc_set_tuning: the tensor-core z transform needs an FP32 context with N <= 128");
    c->z_tc = t->z_transform;
    c->persistent = t->persistent;
    c->overlap = t->overlap;
    c->fft_sched = t->fft_schedule;
    c->spread_mode = t->spread;
    c->sweep_batch = t->sweep_batch;
    c->replay = t->graphs == 1;
    if (!c->replay) c->ws.drop_graph();
    return BC_OK;
}

} // extern "C"

// Median device time (ms) of `reps` calls of fn after `warm` untimed ones,
// each bracketed by events on the context stream.
template <class F>
static bc_status time_median(bc_ctx_t c, F fn, int warm, int reps, float *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "tuning events");
    }
    bc_status s = BC_OK;
    std::vector<float> t;
    for (int i = 0; s == BC_OK && i < warm + reps; i++) {
        if (i >= warm && (e = cudaEventRecord(e0, c->stream)) != cudaSuccess) s = cuda_fail(e, "tuning record");
        if (s == BC_OK) s = fn();
        if (s == BC_OK && i >= warm) {
            float x = 0.f;
            if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&x, e0, e1)) != cudaSuccess)
                s = cuda_fail(e, "tuning timing");
            t.push_back(x);
        }
    }
    if (s == BC_OK) s = bc_sync(c);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != BC_OK) return s;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return BC_OK;
}

extern "C" {

bc_status bc_autotune(bc_ctx_t c, bc_shape_t A, bc_shape_t B, int rotations, bc_tuning *out)
{
    try {
        if (!c || !A || !B) return fail(BC_ERR_ARG, "bc_autotune: null argument");
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_autotune: shapes belong to another context");
        if (rotations < 0 || rotations > 65534) return fail(BC_ERR_ARG, "bc_autotune: rotations must be in [0, 65534]");
        CK(cudaStreamSynchronize(c->stream));
        const long long N3 = (long long)c->g.N * c->g.N * c->g.N;
        cudaError_t e;
        if ((e = c->tune.ensure(sizeof(float) * (size_t)std::max<long long>(N3, 2LL * rotations), false, c->stream)) != cudaSuccess)
            return cuda_fail(e, "bc_autotune: scratch");
        float *dout = (float *)c->tune.p;
        // spreading: one correlation of A with B, unrotated
        static const float ident[4] = {1.f, 0.f, 0.f, 0.f};
        float best = 0.f;
        int best_mode = c->spread_mode;
        for (int mode = 0; mode <= 1; mode++) {
            c->spread_mode = mode;
            float ms = 0.f;
            bc_status s = time_median(c, [&]() { return bc_correlate(c, A, B, ident, 1, dout, 1); }, 3, 7, &ms);
            if (s != BC_OK) {
                c->spread_mode = best_mode;
                return s;
            }
            if (mode == 0 || ms < best) {
                best = ms;
                best_mode = mode;
            }
        }
        c->spread_mode = best_mode;
        // z transform: FFT or tensor-core DFT product (spread 0 only)
        if (c->zdft && c->spread_mode == 0) {
            const int saved = c->z_tc;
            float tz[2] = {0.f, 0.f};
            for (int z = 0; z <= 1; z++) {
                c->z_tc = z;
                bc_status s = time_median(c, [&]() { return bc_correlate(c, A, B, ident, 1, dout, 1); }, 3, 7, &tz[z]);
                if (s != BC_OK) {
                    c->z_tc = saved;
                    return s;
                }
            }
            c->z_tc = tz[1] < tz[0] ? 1 : 0;
        }
        // back half: three launches or one persistent launch
        {
            const int saved = c->persistent;
            float tb[2] = {0.f, 0.f};
            for (int b = 0; b <= 1; b++) {
                c->persistent = b;
                bc_status s = time_median(c, [&]() { return bc_correlate(c, A, B, ident, 1, dout, 1); }, 3, 7, &tb[b]);
                if (s != BC_OK) {
                    c->persistent = saved;
                    return s;
                }
            }
            c->persistent = tb[1] < tb[0] ? 1 : 0;
        }
        // radix schedule per forward pass (the split-precision passes have their own):
        // the stage times of profiled correlations under each schedule, pass by pass
        if (c->g.prec == 0) {
            double stage_ms[2][BC_NUM_STAGES] = {};
            const int saved = c->fft_sched;
            for (int sched = 0; sched <= 1; sched++) {
                c->fft_sched = sched ? 7 : 0;
                bc_status s = BC_OK;
                for (int i = 0; s == BC_OK && i < 3; i++) s = bc_correlate(c, A, B, ident, 1, dout, 1); // warm-up
                bc_profile prof;
                if (s == BC_OK) s = bc_profile_begin(c, 7);
                for (int i = 0; s == BC_OK && i < 7; i++) s = bc_correlate(c, A, B, ident, 1, dout, 1);
                if (s == BC_OK) s = bc_profile_end(c, &prof);
                if (s != BC_OK) {
                    c->fft_sched = saved;
                    return s;
                }
                for (int st = 0; st < BC_NUM_STAGES; st++) stage_ms[sched][st] = prof.ms[st];
            }
            int mask = 0;
            const int stage_of_bit[3] = {2, 3, 4}; // fft_z, fft_y, fft_x
            for (int b = 0; b < 3; b++)
                if (stage_ms[1][stage_of_bit[b]] < 0.98 * stage_ms[0][stage_of_bit[b]]) mask |= 1 << b; // beyond noise
            c->fft_sched = mask;
        }
        if (rotations > 0) {
            // fixed rotations: Shoemake's map of a golden-ratio (Weyl) sequence in [0, 1)^3
            std::vector<float> q(4 * (size_t)rotations);
            for (int r = 0; r < rotations; r++) {
                const double u1 = std::fmod(0.5 + r * 0.6180339887498949, 1.0);
                const double u2 = std::fmod(0.5 + r * 0.7548776662466927, 1.0);
                const double u3 = std::fmod(0.5 + r * 0.5698402909980532, 1.0);
                const double a = std::sqrt(1.0 - u1), b = std::sqrt(u1);
                q[4 * r + 0] = (float)(a * std::sin(2 * M_PI * u2));
                q[4 * r + 1] = (float)(a * std::cos(2 * M_PI * u2));
                q[4 * r + 2] = (float)(b * std::sin(2 * M_PI * u3));
                q[4 * r + 3] = (float)(b * std::cos(2 * M_PI * u3));
            }
            float *dpeak = dout;
            int *darg = (int *)(dout + rotations);
            static const int cand[] = {16, 32, 64, 128, 256};
            int best_batch = c->sweep_batch;
            bool first = true;
            for (int b : cand) {
                if (b > std::max(rotations, 16)) break;
                float ms = 0.f;
                bc_status s = time_median(
                    c, [&]() { return sweep_impl(c, A, B, q.data(), nullptr, rotations, b, dpeak, darg, 1); }, 1, 3, &ms);
                if (s != BC_OK) return s;
                if (first || ms < best) {
                    best = ms;
                    best_batch = b;
                    first = false;
                }
            }
            c->sweep_batch = best_batch;
            // the z transform again, on the sweep itself (its passes batch many
            // rotations of the smaller shape, which can favour the other transform)
            if (c->zdft && c->spread_mode == 0) {
                const int saved = c->z_tc;
                float tz[2] = {0.f, 0.f};
                for (int z = 0; z <= 1; z++) {
                    c->z_tc = z;
                    bc_status s = time_median(
                        c, [&]() { return sweep_impl(c, A, B, q.data(), nullptr, rotations, best_batch, dpeak, darg, 1); },
                        1, 3, &tz[z]);
                    if (s != BC_OK) {
                        c->z_tc = saved;
                        return s;
                    }
                }
                c->z_tc = tz[1] < tz[0] ? 1 : 0;
            }
        }
        if (out) bc_get_tuning(c, out);
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_autotune: unexpected exception");
    }
}

} // extern "C"

// ------------------------------------------------------------------ single-configuration queries
// The first m' modes of the canonical half space -- m_z > 0, or m_z = 0 and
// (m_y > 0, or m_y = 0 and m_x >= 0) -- with components in (-N/2, N/2),
// ordered by (|m|^2, m_x, m_y, m_z); w = 1 for m = 0, 2 otherwise.
static std::vector<std::array<int, 4>> query_modes(int N, int mprime)
{
    const int h = N / 2 - 1; // largest |component|
    int R = (int)std::ceil(std::cbrt(3.0 * mprime / (2.0 * M_PI))) + 2;
    std::vector<std::array<int, 5>> cand;
    for (;;) {
        if (R > h) R = h;
        cand.clear();
        const long long R2 = (long long)R * R;
        for (int mx = -R; mx <= R; mx++)
            for (int my = -R; my <= R; my++)
                for (int mz = 0; mz <= R; mz++) {
                    const long long q = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
                    if (R < h && q > R2) continue;
                    const bool canon = mz > 0 || (my > 0 || (my == 0 && mx >= 0));
                    if (canon) cand.push_back({(int)q, mx, my, mz, 0});
                }
        if ((long long)cand.size() >= mprime || R == h) break;
        R = R * 2;
    }
    std::sort(cand.begin(), cand.end());
    std::vector<std::array<int, 4>> out;
    for (int i = 0; i < mprime && i < (int)cand.size(); i++)
        out.push_back({cand[i][1], cand[i][2], cand[i][3], cand[i][0] == 0 ? 1 : 2});
    return out;
}

extern "C" {

bc_status bc_query_create(bc_ctx_t c, bc_shape_t A, bc_shape_t B, const float *quat, int mprime, bc_query_t *out)
{
    bc_query_s *qo = nullptr;
    try {
        if (!c || !A || !B || !quat || !out) return fail(BC_ERR_ARG, "bc_query_create: null argument");
        *out = nullptr;
        if (A->ctx != c || B->ctx != c) return fail(BC_ERR_ARG, "bc_query_create: shapes belong to another context");
        if (bc_status s = check_quats(quat, 1, "bc_query_create")) return s;
        const int N = c->g.N;
        const long long total = ((long long)(N - 1) * (N - 1) * (N - 1) + 1) / 2;
        if (mprime < 1 || mprime > total)
            return fail(BC_ERR_ARG, "bc_query_create: m' must be in [1, ((N-1)^3 + 1) / 2]");
        const std::vector<std::array<int, 4>> modes = query_modes(N, mprime);
        if ((int)modes.size() != mprime) return fail(BC_ERR_INTERNAL, "bc_query_create: mode enumeration");
        cudaStream_t st = c->stream;
        cudaError_t e;
        qo = new bc_query_s();
        qo->ctx = c;
        qo->count = mprime;
        const size_t spec = sizeof(float2) * (size_t)N * N * c->g.H;
        auto bail = [&](bc_status s) {
            qo->release();
            delete qo;
            return s;
        };
        if ((e = qo->modes.ensure(sizeof(int4) * mprime, false, st)) != cudaSuccess ||
            (e = qo->ghat.ensure(sizeof(float2) * mprime, false, st)) != cudaSuccess ||
            (e = qo->io.ensure(spec, false, st)) != cudaSuccess)
            return bail(cuda_fail(e, "bc_query_create: buffers"));
        if ((e = cudaMemcpyAsync(qo->modes.p, modes.data(), sizeof(int4) * mprime, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(cuda_fail(e, "bc_query_create: modes"));
        // f^_A into the workspace cache, kept in io; then f^_RB into the cache
        std::vector<PairDesc> pairs(1, PairDesc{0, -1, 0, 0, 0});
        if (bc_status s = enqueue(c, std::vector<bc_shape_t>(1, A), std::vector<const float *>(1, nullptr), pairs, true,
                                  nullptr, nullptr))
            return bail(s);
        if ((e = cudaMemcpyAsync(qo->io.p, c->ws.fa.p, spec, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return bail(cuda_fail(e, "bc_query_create: copy spectrum"));
        if (bc_status s = enqueue(c, std::vector<bc_shape_t>(1, B), std::vector<const float *>(1, quat), pairs, true,
                                  nullptr, nullptr))
            return bail(s);
        if ((e = launch_query_gather((const float2 *)qo->io.p, (const float2 *)c->ws.fa.p, (const int4 *)qo->modes.p,
                                     mprime, N, (float2 *)qo->ghat.p, st)) != cudaSuccess)
            return bail(cuda_fail(e, "bc_query_create: gather"));
        if (bc_status s = bc_sync(c)) return bail(s);
        c->queries.insert(qo);
        *out = qo;
        return BC_OK;
    } catch (...) {
        if (qo) {
            qo->release();
            delete qo;
        }
        return fail(BC_ERR_INTERNAL, "bc_query_create: unexpected exception");
    }
}

bc_status bc_query_eval(bc_query_t q, const float *t, int npts, float *g, int on_device)
{
    try {
        if (!q || !t || !g) return fail(BC_ERR_ARG, "bc_query_eval: null argument");
        if (!q->ctx) return fail(BC_ERR_ARG, "bc_query_eval: the query's context was destroyed");
        if (npts < 1 || npts > (1 << 26)) return fail(BC_ERR_ARG, "bc_query_eval: npts must be in [1, 2^26]");
        bc_ctx_t c = q->ctx;
        cudaStream_t st = c->stream;
        cudaError_t e;
        const float *dt = t;
        float *dg = g;
        if (!on_device) {
            const size_t need = sizeof(float) * 4 * (size_t)npts;
            if ((e = q->io.ensure(need, false, st)) != cudaSuccess) return cuda_fail(e, "bc_query_eval: staging");
            float *stage = (float *)q->io.p;
            if ((e = cudaMemcpyAsync(stage, t, sizeof(float) * 3 * (size_t)npts, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(e, "bc_query_eval: copy points");
            dt = stage;
            dg = stage + 3 * (size_t)npts;
        }
        if ((e = launch_query_eval((const float2 *)q->ghat.p, (const int4 *)q->modes.p, q->count, c->g.N, c->period, dt,
                                   npts, dg, st)) != cudaSuccess)
            return cuda_fail(e, "bc_query_eval: launch");
        if (!on_device) {
            if ((e = cudaMemcpyAsync(g, dg, sizeof(float) * (size_t)npts, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_fail(e, "bc_query_eval: copy results");
            CK(cudaStreamSynchronize(st));
        }
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_query_eval: unexpected exception");
    }
}

bc_status bc_query_destroy(bc_query_t q)
{
    if (!q) return BC_OK;
    try {
        if (q->ctx) {
            cudaStreamSynchronize(q->ctx->stream);
            q->ctx->queries.erase(q);
        }
        q->release();
        delete q;
        return BC_OK;
    } catch (...) {
        return fail(BC_ERR_INTERNAL, "bc_query_destroy: unexpected exception");
    }
}

} // extern "C"
