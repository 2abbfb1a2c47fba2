// Internal declarations shared by the C-ABI layer (bc_api.cu) and the kernels
// (bc_kernels.cu).  Not part of the public interface.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

struct bc_ctx_s;
struct bc_mlp_s;

namespace bc {

// Per-instance description: one shape (A, or B under one rotation) whose
// spectrum is computed in this launch.  Built on the host, read on the device.
struct InstDesc {
    int knot_off;       // first knot of this instance in the prepared-knot array
    int nknots;         // knot count
    int src_off;        // first knot of its shape in the shape's knot array (always 0)
    int cap_e;          // per-axis capacity of the compact spreading box
    long long grid_off; // float offset of its spreading boxes (L boxes)
    long long z1_off;   // float2 offset of its z-transformed planes
    long long y1_off;   // float2 offset of its y-transformed planes
    float q[4];         // rotation (w, x, y, z), unit; identity for A
    const float4 *knots; // the shape's knots (x, y, z, level bits)
    const float *qdev;   // when not null: the rotation is read from this device address instead of q
};

// Device-computed support box of one instance in fine-grid cells.
struct InstPlan {
    int lo[3]; // first cell (may be negative: cells are centred on the origin)
    int b[3];  // extent per axis (0 = empty instance)
    int pos0[3]; // lo mod n: where compact index 0 lands in a length-n line
    int bzp;   // z extent padded to a multiple of 4
};

// A correlation output: the spectra of instances a and b are combined into
// out[...] (a < 0: use the cached spectrum of A).
struct PairDesc {
    int a, b;
    long long h_off;    // float2 offset of this pair's inverse-transform planes
    long long out_off;  // float offset of this pair's output grid (when a grid is written)
    long long key;      // slot of this pair's peak key (when peaks are taken)
};

struct Tables {
    const float *deconv;  // N: 1 / phi^(m/n), m in FFT order
    const float *ballft;  // L x (3 (N/2)^2 + 1): h^(rho_l, 2 pi sqrt(q) / P), q = |m|^2
    const float2 *tw_n;   // n twiddles exp(-2 pi i k / n)
    const float2 *tw_N;   // N twiddles exp(-2 pi i k / N)
    int qmax;             // 3 (N/2)^2
    const float *consts;  // [0] = exp(beta) / I0(beta), the window normalisation
    // x-pass level weights, per (j_y, chunk of 16 z-modes) one contiguous slice
    // [l][a = |m_x| in 0..N/2][16]: ballft_l(a^2 + m_y^2 + m_z^2) D(a) D(m_y) D(m_z)
    // (null: the x pass builds them from ballft and deconv)
    const float *xw;
};

struct Geometry {
    int N, n, W, L, H;  // H = N/2 kept z modes
    float beta, n_over_P, inv_P3;
    int prec;           // 0: FP32 transforms; 1: radix-8 stages as split BF16 tensor-core DFTs
    int sched;          // alternative radix schedule for the forward FP32 passes: bit 0 z, bit 1 y, bit 2 x
    int pdl;            // 1: the passes after k_prepare launch as programmatic dependents of the one before
};

// Kernel launchers (bc_kernels.cu).  All return cudaGetLastError() after launch.
cudaError_t launch_build_tables(const Geometry &g, double beta, double period, const double *radii_dev,
                                float *deconv, float *ballft, float2 *tw_n, float2 *tw_N, float *consts,
                                cudaStream_t s);
// out[l][q] = h^(rho_l + r0, k) - lambda h^(rho_l, k), k = 2 pi sqrt(q) / P (FP64, rounded once).
// The x-pass weight table of Tables::xw from `ballft` (N (N/32) L (N/2 + 1) 16 floats).
cudaError_t launch_build_xw(const Geometry &g, const float *deconv, const float *ballft, float *xw, cudaStream_t s);
size_t xw_floats(const Geometry &g);
cudaError_t launch_build_score_table(const Geometry &g, double period, const double *radii_dev, double r0,
                                     double lambda, float *out, cudaStream_t s);
cudaError_t launch_pack_knots(const float *xyz, const int *level, int n, int L, float4 *knots,
                              unsigned int *stats, cudaStream_t s);
// bb: 8 ints per instance (support-box accumulators); they must hold the reset
// state (launch_reset_boxes) before the first launch and are left reset.
cudaError_t launch_reset_boxes(int *bb, int ninst, cudaStream_t s);
// With cnt (ninst * L * n zeroed ints) the knots are also counted per bin
// (instance, level, first stencil cell along x mod n) and the counts turned
// into bin cursors cur (same size; cnt is left zeroed) for launch_bin.
cudaError_t launch_prepare(const Geometry &g, const InstDesc *inst, int ninst, int max_knots, float4 *ku, int *bb,
                           InstPlan *plan, int *err, int *cnt, int *cur, cudaStream_t s);
// Binned spreading (bc_binned.cu).  cur[b] = first slot of bin b (the
// instance's knot_off plus the counts of the bins before it in the instance);
// launch_bin writes one BIN_REC-float record per knot into its bin (cur[b] is
// then the end of bin b); launch_fft_z_binned spreads each z-transform item's
// knots in shared memory and transforms them (no spreading grid in HBM).
constexpr int MAX_W = 10;   // widest window (bc_create checks)
// Tables::consts: [0] = exp(beta) / I0(beta); from [KB_OFF], per stencil offset
// t < W, the KB_NC coefficients of the window's piecewise polynomial (see
// kb_poly in bc_device.cuh).
constexpr int KB_DEG = 10, KB_NC = KB_DEG + 1, KB_OFF = 4;
constexpr int CONSTS_FLOATS = KB_OFF + MAX_W * KB_NC;
constexpr int BIN_REC = 32; // floats per binned knot: g0_y, g0_z (int bits), W x-, W y-, W z-weights
// Plans each instance (as launch_prepare does without bins) and turns the counts
// into cursors, one block per instance.
cudaError_t launch_plan_bins(const Geometry &g, const InstDesc *inst, int ninst, int *bb, InstPlan *plan, int *err,
                             int *cnt, int *cur, cudaStream_t s);
cudaError_t launch_bin(const Geometry &g, const Tables &t, const InstDesc *inst, int total_knots, const float4 *ku,
                       const InstPlan *plan, int *cur, float *rec, cudaStream_t s);
cudaError_t launch_fft_z_binned(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                                const InstPlan *plan, const int *cur, const float *rec, float2 *z1, int nsm,
                                cudaStream_t s);
cudaError_t launch_spread(const Geometry &g, const Tables &t, const InstDesc *inst, int total_knots,
                          const float4 *ku, const InstPlan *plan, float *grid, int nsm, cudaStream_t s);
cudaError_t launch_fft_z(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                         const InstPlan *plan, float *grid, float2 *z1, int nsm, cudaStream_t s);
// The z pass as split-TF32 DFT products on the tensor cores (bc_zumma.cu),
// N in {32, 64, 96, 128} with n = 2N: same output as launch_fft_z, boxes left
// cleared; a stalled wait sets bit 8 of *err.  bhi / blo: the 32-cell DFT block
// from launch_build_zdft (n/2 x 32 floats each).
bool supported_z_umma(int N);
// One thread waits (bounded) on an mbarrier nothing arrives at: sets bit 8 of *err.
cudaError_t launch_wait_selftest(int *err, cudaStream_t s);
cudaError_t launch_build_zdft(int n, float *bhi, float *blo, cudaStream_t s);
cudaError_t launch_fft_z_umma(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                              const InstPlan *plan, float *grid, float2 *z1, const float *bhi, const float *blo,
                              int *err, int nsm, cudaStream_t s);
// max_cap: the largest per-axis box capacity (InstDesc::cap_e) of the instances;
// when it is small enough the pass stages each item's rows from position 0.
cudaError_t launch_fft_y(const Geometry &g, const Tables &t, const InstDesc *inst, int ninst,
                         const InstPlan *plan, const float2 *z1, float2 *y1, int max_cap, int nsm, cudaStream_t s);
cudaError_t launch_fft_x(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                         const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache,
                         float2 *fa_out, float2 *h, int nsm, cudaStream_t s);
// The x, inverse-y and inverse-z passes of pairs (all with b >= 0) as one
// persistent launch over a device work queue (bc_back.cu); `sync` holds
// back_sync_words(N, npairs) counters, cleared by the launcher.  An expired
// dependency wait sets bit 4 of *err.
size_t back_sync_words(int N, int npairs);
// One block waits (bounded) on a counter nothing raises (`zeroed` is cleared
// first): sets bit 4 of *err after about two seconds.
cudaError_t launch_queue_wait_selftest(unsigned *zeroed, int *err, cudaStream_t s);
cudaError_t launch_back(const Geometry &g, const Tables &t, const InstDesc *inst, const InstPlan *plan,
                        const PairDesc *pairs, int npairs, const float2 *y1, const float2 *fa_cache, float2 *h,
                        float *out, unsigned long long *keys, unsigned *sync, int *err, int nsm, cudaStream_t s);
cudaError_t launch_ifft_y(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, float2 *h,
                          int nsm, cudaStream_t s);
// out (N^3 floats per pair) and keys (one 64-bit peak key per pair slot) may each be null.
cudaError_t launch_ifft_z(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs,
                          const float2 *h, float *out, unsigned long long *keys, int nsm, cudaStream_t s);
// The inverse y and z passes of whole planes in shared memory, one block per
// plane (N <= 128): the same result as launch_ifft_y then launch_ifft_z, for
// batches of many pairs.
cudaError_t launch_ifft_yz(const Geometry &g, const Tables &t, const PairDesc *pairs, int npairs, const float2 *h,
                           float *out, unsigned long long *keys, int nsm, cudaStream_t s);
// keys[i] -> peak[i], argmax[i] (i < n).
cudaError_t launch_decode_peaks(const unsigned long long *keys, int n, float *peak, int *argmax, cudaStream_t s);

bool supported_N(int N);
bool supported_split(int N); // N for which precision 1 is built

// Sets the calling thread's message returned by bc_last_error() (bc_api.cu).
void set_last_error(const std::string &msg);

// Context accessors for the other translation units (bc_api.cu).
cudaStream_t ctx_stream(bc_ctx_s *c);
int *ctx_err(bc_ctx_s *c);
// Networks are registered with their context; destroying the context orphans
// them (their device memory is freed and their context pointer cleared).
void ctx_register_mlp(bc_ctx_s *c, bc_mlp_s *net);
void ctx_unregister_mlp(bc_ctx_s *c, bc_mlp_s *net);
void mlp_orphan(bc_mlp_s *net); // bc_mlp.cu

// Single-configuration queries (bc_query.cu).  modes[i] = (m_x, m_y, m_z, w).
cudaError_t launch_query_gather(const float2 *fa, const float2 *fb, const int4 *modes, int count, int N, float2 *ghat,
                                cudaStream_t s);
cudaError_t launch_query_eval(const float2 *ghat, const int4 *modes, int count, int N, double period, const float *t,
                              int npts, float *g, cudaStream_t s);

// Learned-proposal helpers (bc_mlp.cu).
cudaError_t launch_topk(const float *scores, int n, int k, int *idx, cudaStream_t s);
cudaError_t launch_gather_quats(const float *q, const int *idx, int k, float *out, cudaStream_t s);
// out_i = sq * q_i (sq: 4 host floats, q and out: n x 4 device floats)
cudaError_t launch_compose_quats(const float *sq, const float *q, int n, float *out, cudaStream_t s);
// y = alpha y + beta x (device, n)
cudaError_t launch_axpby(float *y, const float *x, int n, float alpha, float beta, cudaStream_t s);
// out[i] = |F(m_i)| / F(0) for the modes[i] = (m_x, m_y, m_z), i < count, of a cached half spectrum.
cudaError_t launch_moments(const float2 *F, const int *modes, int count, int N, int H, float *out, cudaStream_t s);
// out[r][i] = |f^_S(R_r^T m_i)| / f^_S(0) for the BC_MOMENTS lowest modes m_i and
// the n rotations R_r of `quats` (device, n x 4), by direct sums over the nk knots
// (x, y, z, level bits) with the ball transforms ballft[l (qstride) + |m|^2]; a zero
// quaternion raises bit 4 of *err.
cudaError_t launch_moments_rot(const float4 *knots, int nk, const float *quats, int n, const float *ballft, int qstride,
                               int L, float two_over_P, float *out, int *err, cudaStream_t s);
// Whether the compiled mode table of launch_moments_rot equals `tab` (3 BC_MOMENTS ints).
bool moments_rot_table_matches(const int *tab);

} // namespace bc
