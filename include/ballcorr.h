/*
 * ballcorr: Fourier-domain translational correlation of two unions of balls on
 * an NVIDIA GB300 (sm_103a).  C ABI; no C++ or framework types cross it.
 *
 * What it computes (Behandish & Ilies, "Analytic methods for geometric modeling
 * via spherical decomposition"):
 *
 *   A shape X is a set of knots c_j (centres) with radii drawn from L levels
 *   rho_1..rho_L; its defining function is the sum of the ball indicators
 *   (Eq. (un), Sec. 2.1; the alpha -> infinity limit of Eq. (psi), Sec. 2.2).
 *   Per level the knots form the impulse density of Eq. (rhoP), whose
 *   transform is the nonequispaced sum of Eq. (rhoPhat) (Sec. 2.5):
 *       S_{X,l}(m) = sum_{j in level l} exp(-2 pi i m . x_j / P).
 *   The shape spectrum is the level sum of Eq. (fballhat):
 *       f^_X(m) = sum_l h^(rho_l, k) S_{X,l}(m),  h^(r,k) = 4 pi (sin kr - kr cos kr)/k^3,
 *       k = 2 pi |m| / P,
 *   and the correlation of A with B rotated by R (Eq. (relg), Sec. 3.1) is, in
 *   the Fourier domain, Eq. (ccghat) (Sec. 3.2):
 *       g^(m) = f^_A(m) conj(f^_{RB}(m)),
 *       g(t)  = P^-3 sum_m g^(m) exp(+2 pi i m . t / P)   (App. C).
 *   Modes m lie in [-N/2, N/2)^3; modes with a component equal to -N/2 are
 *   zero, so g is real.  g is sampled on t_k = -P/2 + k P/N, k = 0..N-1 per
 *   axis, and is periodic with period P (knots outside [-P/2, P/2) wrap).
 *
 * How: each level's S_{X,l} is a type-1 nonuniform FFT (Kaiser-Bessel
 * spreading onto a sigma*N oversampled grid, a 3D FFT, division by the window
 * transform); the window division, the ball transform, the level sum, the
 * conjugate product and the inverse transform run in fused CUDA kernels.
 * Floating point work is FP32; the window and ball-transform tables are built
 * in FP64 on the device and rounded once.
 *
 * Conventions for every call:
 *   - Every function returns a bc_status; nothing throws across the ABI.
 *     bc_last_error() gives a message for the calling thread's last failure.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous unless
 *     a host buffer is involved (then the call synchronises that stream).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - Caller-owned buffers stay caller-owned; the library copies what it keeps
 *     and owns all of its internal workspaces.
 *   - A context (and everything created on it) is used by one host thread at
 *     a time; different contexts may be used from different threads.  The
 *     calling thread's current CUDA device must be the one that was current
 *     when the context was created (a new host thread starts on device 0).
 */
#ifndef BALLCORR_H
#define BALLCORR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bc_ctx_s *bc_ctx_t;
typedef struct bc_shape_s *bc_shape_t;

typedef enum {
    BC_OK = 0,
    BC_ERR_ARG = 1,         /* invalid argument (sizes, pointers, level id, zero quaternion) */
    BC_ERR_OOM = 2,         /* device allocation failed */
    BC_ERR_CUDA = 3,        /* a CUDA call failed; see bc_last_error() */
    BC_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired */
    BC_ERR_UNSUPPORTED = 5, /* parameters outside what this build supports */
    BC_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} bc_status;

#define BC_MAX_LEVELS 8

/* Correlation parameters.  Supported: N in {32, 64, 96, 128, 256}, sigma = 2
 * (so the oversampled grid has n = 2N points per axis), 2 <= W <= 10.
 * beta is rounded to FP32 once; the window and its FP64 transform table both
 * use that rounded value. */
typedef struct {
    int N;                     /* modes per axis = translation samples per axis */
    int sigma;                 /* oversampling factor of the spreading grid (2) */
    int W;                     /* Kaiser-Bessel window width in fine-grid cells */
    double beta;               /* window shape; <= 0 selects pi*sqrt((W/sigma)^2 (sigma-1/2)^2 - 0.8) */
    double period;             /* P > 0: the translation grid covers [-P/2, P/2)^3 */
    int level_count;           /* L, 1..BC_MAX_LEVELS */
    const double *level_radii; /* host array of L radii (> 0); copied */
    int precision;             /* 0 = FP32; 1 = the radix-8 stages of the forward transforms run as
                                  BF16 hi+lo split DFT matmuls on the tensor cores with FP32
                                  accumulation (radix schedules with radix-8 stages: 64 = 8.8,
                                  128 = 8.16, 192 = 3.8.8, 256 = 4.8.8, 512 = 8.8.8; every N) */
} bc_params;

/* Creates a context on the current CUDA device bound to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Builds the window,
 * ball-transform and twiddle tables.  Errors: BC_ERR_ARG (null pointer,
 * parameters out of range), BC_ERR_UNSUPPORTED, BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_create(const bc_params *params, void *cuda_stream, bc_ctx_t *out);

/* Synchronises the context stream and frees everything it owns, including the
 * device memory of shapes still alive on it (their handles stay valid only for
 * bc_shape_destroy).  NULL is accepted. */
bc_status bc_destroy(bc_ctx_t ctx);

/* Uploads a shape: n knots, xyz = n x 3 FP32 centres (row major), level = n
 * level ids in [0, L).  `on_device` says whether both arrays are device (1) or
 * host (0) memory.  The library copies them; the caller keeps its arrays.
 * Synchronises the context stream (it validates levels and sizes workspaces).
 * n = 0 gives an empty shape, whose correlation with anything is 0.
 * Errors: BC_ERR_ARG (null pointer with n > 0, n < 0, level out of range,
 * non-finite coordinate), BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_shape_create(bc_ctx_t ctx, const float *xyz, const int *level, int n, int on_device,
                          bc_shape_t *out);

/* Uploads `count` shapes with one stream synchronisation for all of them
 * (bc_shape_create is the count = 1 case): shape i has n[i] knots with
 * centres xyz[i] and level ids level[i], arrays as in bc_shape_create, all
 * device (on_device = 1) or all host (0) memory; out[i] receives its handle.
 * Host arrays in page-locked memory mapped into the device address space are
 * read by the packing kernel directly; other host arrays are staged on the
 * device first.
 * On any error no shape is created (every out[i] is NULL) and the message
 * names the first failing shape.  Errors as bc_shape_create, and BC_ERR_ARG
 * for count < 0 or null arrays. */
bc_status bc_shapes_create(bc_ctx_t ctx, int count, const float *const *xyz, const int *const *level, const int *n,
                           int on_device, bc_shape_t *out);

/* Frees a shape (stream-ordered after pending work on the context).  NULL is accepted.
 * A shape whose context was destroyed first has already lost its device memory;
 * this call then only releases the handle. */
bc_status bc_shape_destroy(bc_shape_t shape);

/* g(R_q, t) for k rotations of B:  out[r][kx][ky][kz] = g(R(q_r), t_k), an
 * FP32 array of k * N^3 values, kz fastest.  quats: k x 4 FP32 (w, x, y, z),
 * normalised internally, host memory.  A is not rotated.  `out_on_device`
 * selects device (1, asynchronous) or host (0, synchronous) output memory.
 * A host `out` in page-locked memory mapped into the device address space
 * (cudaMallocHost, cudaHostAlloc, cudaHostRegister) is written by the last
 * kernel directly; other host memory is staged on the device and copied.
 * Errors: BC_ERR_ARG (k < 1, null pointer, zero quaternion, shapes from
 * another context), BC_ERR_OOM, BC_ERR_CUDA, BC_ERR_INTERNAL. */
bc_status bc_correlate(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quats, int k,
                       float *out, int out_on_device);

/* Rotation sweep: for each of k rotations of B, the peak of the correlation
 * over the translation grid,
 *     peak[r]   = max_t g(R(q_r), t),
 *     argmax[r] = the lowest linear index (kx*N + ky)*N + kz attaining it,
 * without writing the N^3 grids.  A's spectrum is computed once per call and
 * reused; the rotations run in batches of `batch` (0 = the context's
 * sweep_batch, see bc_set_tuning) through the same
 * kernels as bc_correlate, the last of which folds each batch's grids into
 * 64-bit peak keys.  quats: k x 4 FP32 host memory.  peak (k floats) and
 * argmax (k ints) are device (out_on_device = 1, asynchronous) or host
 * (0, synchronous) memory.  Errors: BC_ERR_ARG (null pointer, k < 1, zero
 * quaternion, shapes from another context), BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_sweep(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, float *peak,
                   int *argmax, int out_on_device);

/* Captured sweep: the whole of bc_sweep(ctx, A, B, quats, k, batch, peak,
 * argmax, 1) -- clearing the peak keys, A's spectrum, every batch of rotations
 * and the decoding -- recorded once as a CUDA graph over workspaces the plan
 * owns, so that each bc_plan_run is a single graph launch on ctx's stream.
 * quats (host) are copied at plan time; peak and argmax are device buffers
 * fixed at plan time; A and B must outlive the plan.  Planning synchronises
 * the stream.  Errors as bc_sweep, plus BC_ERR_CUDA from graph capture. */
typedef struct bc_plan_s *bc_plan_t;
bc_status bc_sweep_plan(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, float *peak,
                        int *argmax, bc_plan_t *out);
bc_status bc_plan_run(bc_plan_t plan);
bc_status bc_plan_destroy(bc_plan_t plan);

/* Ragged batch of independent pairs: pair i correlates As[i] with Bs[i]
 * rotated by quats[i] (npairs x 4 FP32, host).  Shapes may have any knot
 * counts; every instance gets its own support box.  Outputs (either may be
 * NULL, not both): out[i][kx][ky][kz] (npairs * N^3 floats) and
 * peak[i] / argmax[i] as in bc_sweep.  All output pointers are device memory
 * (on_device = 1, asynchronous) or host memory (0, synchronous); a host `out`
 * is written as bc_correlate's.
 * Errors: BC_ERR_ARG (null shape or quaternion array, zero quaternion, both
 * outputs null, peak without argmax, npairs outside [1, 32767], shapes from
 * another context), BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_pairs(bc_ctx_t ctx, const bc_shape_t *As, const bc_shape_t *Bs, const float *quats, int npairs,
                   float *out, float *peak, int *argmax, int on_device);

/* ---------------------------------------------------------------- shape complementarity
 * Score of Sec. 4.2, Eq. (score): with the affinity F_S = i (f_{S+B0} -
 * lambda f_S) (S + B0 the offset of S by the ball of radius r0, which for a
 * union of balls is the same knots with every radius grown by r0) and the
 * correlation of the two affinity functions taken without conjugation,
 *     G(R, t) = -lambda^2 g_{A,RB}(t) + lambda g_{A+B0,RB}(t)
 *               + lambda g_{A,RB+B0}(t) - g_{A+B0,RB+B0}(t),
 * i.e. a penalty for core-core overlap, a reward for offset-core overlap and
 * a smaller penalty for offset-offset overlap (the signs the paper's text
 * gives the three terms of its expansion).  Computed as one band-limited
 * correlation whose per-level multiplier is h^(rho_l + r0, k) -
 * lambda h^(rho_l, k) (built in FP64 for each new (r0, lambda)) and whose
 * product is negated.  bc_score has the layout, memory and error behaviour of
 * bc_correlate, bc_score_sweep those of bc_sweep (peak = max_t G).
 * Errors additionally: BC_ERR_ARG when r0 or lambda is negative or not finite. */
bc_status bc_score(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quats, int k, double r0, double lambda,
                   float *out, int out_on_device);
bc_status bc_score_sweep(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quats, int k, int batch, double r0,
                         double lambda, float *peak, int *argmax, int out_on_device);

/* ---------------------------------------------------------------- single-configuration queries
 * Time-critical evaluation at arbitrary translations (Sec. 4.1, Eq. (single)):
 * the inner product of f_A with f_RB shifted by t is, by Parseval, a sum over
 * the modes of g^ = f^_A conj(f^_RB) (Eq. (ccghat)), which is truncated to
 * the m' modes nearest the origin -- the traversal of the frequency grid
 * outward from the dominant low modes --
 *     g'(R, t) = P^-3 sum_{m in M'} w_m Re( g^(m) exp(2 pi i m.t / P) ),
 * M' = the first m' modes of the canonical half space (m_z > 0, or m_z = 0 and
 * (m_y > 0, or m_y = 0 and m_x >= 0)) with components in (-N/2, N/2), ordered
 * by (|m|^2, m_x, m_y, m_z); w_m = 1 for m = 0 and 2 otherwise (the mode and
 * its conjugate -m).  With m' = ((N-1)^3 + 1) / 2 (all modes) g' is the
 * band-limited correlation itself, at any t; a collision predicate is g' > 0.
 *
 * bc_query_create computes both spectra once (the pipeline of bc_correlate up
 * to the spectra; quat: 4 FP32 host values) and keeps g^ at the m' modes.
 * Synchronous.  Errors: BC_ERR_ARG (null pointer, zero quaternion, shapes from
 * another context, m' outside [1, ((N-1)^3 + 1) / 2]), BC_ERR_OOM, BC_ERR_CUDA.
 * bc_query_eval: t = npts x 3 FP32 translations, g = npts FP32 results, both
 * device (on_device = 1, asynchronous on ctx's stream) or host (0,
 * synchronous) memory; any t is allowed (g' is P-periodic).  Errors:
 * BC_ERR_ARG (null pointer, npts outside [1, 2^26], context destroyed),
 * BC_ERR_CUDA.  bc_query_destroy waits for the context stream. */
typedef struct bc_query_s *bc_query_t;
bc_status bc_query_create(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, const float *quat, int mprime, bc_query_t *out);
bc_status bc_query_eval(bc_query_t q, const float *t, int npts, float *g, int on_device);
bc_status bc_query_destroy(bc_query_t q);

/* ---------------------------------------------------------------- lifted (4D) correlation
 * Nonequiradius correlation of Sec. 3.2 (Eqs. (L2cone), (rhoA), (rhoAhat),
 * (fconehat), (convgA); Lemma 2) for knots with individual radii.  Knot
 * (x, r) lifts to the trimmed half-cone D(x, r) = {(y, s) : |y - x| <= r - s,
 * r - L <= s <= r}, whose s = 0 section is the ball of radius r; B is rotated
 * and then mirrored in r (s -> -s), and the lifted correlation g(t, r) is the
 * correlation of the two cone unions' indicator sums at the lifted translation
 * (t, r): the summed 4D overlap volume of the cone pairs.  Its r = 0 section
 * is positive exactly at the translations where a ball of A meets a ball of
 * t + RB (Lemma 2); a section r != 0 is the obstacle of the shapes offset by
 * a total of -r.  Computed by a direct 4D NDFT (Eq. (rhoAhat)) on the modes
 * xi in [-N/2, N/2)^3, eta in [-Nr/2, Nr/2) (lower-edge modes zero), times the
 * squared cone transform f^_D0 (FP64-built table), then for each requested
 * section the sum over eta and the inverse 3D transform onto the N^3 grid
 * t_k = -P/2 + k P/N:
 *     g(t, r) = P^-3 P_r^-1 sum g^(xi, eta) exp(2 pi i (xi . t / P + eta r / P_r)),
 *     g^      = rho^_A conj(rho^_{RB mirrored}) f^_D0^2.
 * Radii should lie in (0, L) (every cone reaches s = 0) and P_r should exceed
 * 4 L so that sections do not wrap.  Not in the correlation context: a lifted
 * context owns its tables and workspace.
 * bc_lift_correlate: A, B = n x 4 FP32 (x, y, z, r), quat = 4 FP32 host values,
 * slices = nslices (1 .. 16) FP32 host values r_s, out = nslices x N^3 FP32
 * ([s][kx][ky][kz]); A, B and out are device (on_device = 1) or host (0)
 * memory.  Synchronous.  The tensor-core contractions take the knots in
 * passes of 32,768 (their operands cost 16 N^2 + 16 N Nr bytes per knot), so
 * the workspace stays bounded for any knot count.  Errors: BC_ERR_ARG (null pointer, counts out of
 * range, zero quaternion, non-finite section), BC_ERR_UNSUPPORTED (N not 32,
 * 64, 96 or 128, Nr not 8, 16, 32 or 64, Nr = 8 with contraction 3),
 * BC_ERR_OOM, BC_ERR_CUDA, BC_ERR_TIMEOUT (a
 * bounded wait inside the tcgen05 contraction expired; out is incomplete). */
typedef struct bc_lift_s *bc_lift_t;
typedef struct {
    int N;           /* modes per axis and translation grid N^3: 32, 64, 96 or 128 */
    int Nr;          /* modes along the lifted axis: 8, 16, 32 or 64 */
    double L;        /* cone height */
    double period;   /* P, translation period */
    double period_r; /* P_r, period along the lifted axis */
    int contraction; /* how rho^ of Eq. (rhoAhat) is computed, all at FP32-level accuracy:
                        2 direct 4D NDFT on the tcgen05.mma tensor cores (accumulators in
                          tensor memory, operands staged by bulk copies), 3-pass split TF32;
                        1 direct 4D NDFT on the mma.sync tensor cores, 3-pass split TF32;
                        0 direct 4D NDFT in FP32 on the CUDA cores;
                        3 4D type-1 NUFFT: Kaiser-Bessel spreading (width 8) of the lifted
                          knots onto the (2N)^3 x 2Nr grid, a 4D FFT keeping the modes
                          above, deconvolution, the collapse formed from the two
                          spectra directly (Nr >= 16; workspace 52 x 2Nr x N^3 bytes) */
} bc_lift_params;
bc_status bc_lift_create(const bc_lift_params *params, void *cuda_stream, bc_lift_t *out);
bc_status bc_lift_correlate(bc_lift_t lift, const float *A, int nA, const float *B, int nB, const float *quat,
                            const float *slices, int nslices, float *out, int on_device);
bc_status bc_lift_destroy(bc_lift_t lift);

/* ---------------------------------------------------------------- tuning
 * Not in the paper: implementation choices that change speed, not results
 * (beyond the FP32 rounding order of the spreading sums).
 *   spread       0: every knot's W^3 stencil is added to its level's spreading
 *                   box in device memory with global vector atomics, and the
 *                   z transform reads the boxes back;
 *                1: the knots are sorted into bins by their first stencil cell
 *                   along x, and each z-transform item (level, x-cell, 32
 *                   y-rows) adds the (y, z) stencil columns of the knots that
 *                   reach it in shared memory before transforming them; no
 *                   spreading box is kept in device memory.
 *   sweep_batch  rotations per pass of bc_sweep, bc_sweep_plan and
 *                bc_learned_sweep when their batch is 0 (1 .. 65534).
 *   fft_schedule bit mask of the forward FP32 passes (1: z, 2: y, 4: x) that
 *                use an alternative radix schedule (64 = 4.16, 128 = 16.8,
 *                192 = 3.4.16, 256 = 4.8.8, 512 = 8.4.16) instead of the default
 *                of their length (32 = 4.8, 64 = 8.8, 96 = 3.4.8, 128 = 8.16,
 *                192 = 3.8.8, 256 = 16.16, 512 = 8.8.8); 0 .. 7.  Same
 *                transform, other rounding order.
 *   graphs       1: a pass of a direct call (bc_correlate, bc_score, bc_pairs,
 *                ...) whose descriptors, output buffers and workspaces equal
 *                those of the previous pass is replayed from a CUDA graph
 *                recorded on its first run (one graph launch instead of the
 *                kernel launches); 0: always launch kernel by kernel.  Passes
 *                recorded by bc_profile_begin always launch kernel by kernel.
 *   z_transform  with spread 0: 0 the z pass is the radix FFT above; 1 it is a
 *                pruned DFT on the 5th-generation tensor cores: each z line's
 *                bz box cells times the fixed n-point DFT matrix restricted to
 *                m_z in [0, N/2) (tcgen05.mma, 3-pass split TF32, FP32
 *                accumulation restarted every 32 cells), then the phase of the
 *                box origin.  Same transform, other rounding order.  Available
 *                in FP32 contexts with N <= 128 (BC_ERR_UNSUPPORTED otherwise);
 *                a stalled tensor-core wait is reported by bc_sync as
 *                BC_ERR_TIMEOUT.
 *   persistent   0: the x pass (with the deconvolution, ball transforms, level
 *                sum and conjugate product), the inverse y pass and the
 *                inverse z pass run as three launches; 1: one persistent
 *                launch whose blocks take the three passes' work units from a
 *                device queue in order, each unit waiting (bounded, two
 *                seconds; bc_sync reports an expired wait as BC_ERR_TIMEOUT)
 *                for the units it reads to finish.  Same arithmetic.
 *   overlap      1: every pass after the first of a correlation is launched
 *                as a programmatic dependent of the pass before it, so its
 *                blocks take the SMs the earlier pass leaves and run their
 *                set-up (constant tables, tensor memory, barriers) while the
 *                earlier pass finishes; each waits for the earlier pass to
 *                complete before it reads what that pass wrote.  0: each pass
 *                is launched after the previous one has ended.  Same
 *                arithmetic.
 * A new context starts with {0, 64, 1, 0, 1, 0, 1} (z_transform 0 where 1 is
 * not available).  Plans keep the choices in force when
 * they were made.  bc_autotune times the candidates on the given shapes --
 * bc_correlate of A with B (identity) for `spread`, `z_transform` and `persistent` (when rotations > 0,
 * `z_transform` is decided again on the sweep with the chosen batch); in FP32 contexts the
 * per-stage times of profiled correlations under each schedule, pass by pass,
 * for `fft_schedule`; when rotations > 0, a sweep of that many fixed rotations
 * of B for each sweep_batch in {16, 32, 64, 128, 256} not above it -- keeps
 * the fastest in the context and returns them in out (may be NULL).  It
 * synchronises the stream, grows the context's workspaces to the largest
 * candidate and ends any profiling started with bc_profile_begin; it leaves
 * `graphs` and `overlap` as they are.  Errors: BC_ERR_ARG (null context
 * or shape, shapes from another context, rotations outside [0, 65534], a
 * value out of range in bc_set_tuning), BC_ERR_OOM, BC_ERR_CUDA. */
typedef struct {
    int spread;
    int sweep_batch;
    int graphs;
    int fft_schedule;
    int z_transform;
    int persistent;
    int overlap;
} bc_tuning;
bc_status bc_get_tuning(bc_ctx_t ctx, bc_tuning *out);
bc_status bc_set_tuning(bc_ctx_t ctx, const bc_tuning *t);
bc_status bc_autotune(bc_ctx_t ctx, bc_shape_t A, bc_shape_t B, int rotations, bc_tuning *out);

/* ---------------------------------------------------------------- learned proposal
 * Not in the paper: a small network ranks rotations so that only the best
 * ranked ones get full correlations.  Features of a (rotation, pair):
 * x = [q / |q| with w >= 0 (4); m_A (BC_MOMENTS); m_B (BC_MOMENTS)], where
 * m_S[i] = |f^_S(m_i)| / f^_S(0) over the BC_MOMENTS lowest modes of the half
 * spectrum (m_z >= 0, m != 0, components inside (-N/2, N/2)) ordered by
 * (|m|^2, m_x, m_y, m_z), for the unrotated shape -- or, for a network set to
 * take them (bc_mlp_set_features), m_B of the ligand turned by the rotation,
 * m_{R B}[i] = |f^_B(R^T m_i)| / f^_B(0).  Network: 132 -> H -> H -> 1,
 * ReLU, FP32 master weights, BF16 operands on the tensor cores with FP32
 * accumulation, mean squared error, Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameter layout (FP32): W1 [H][132], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]. */
#define BC_MOMENTS 64
#define BC_MLP_IN 132
#define BC_TOPK_MAX 16384
typedef struct bc_mlp_s *bc_mlp_t;

/* out (device, BC_MOMENTS floats) = m_S as above.  Computes S's spectrum with
 * the correlation kernels (overwrites the context's cached spectrum).
 * Errors: BC_ERR_ARG (null pointer, empty shape, foreign shape), BC_ERR_CUDA. */
bc_status bc_shape_moments(bc_ctx_t ctx, bc_shape_t shape, float *out);

/* out (device, n x BC_MOMENTS floats): row r = the moments of the shape turned
 * by rotation r of quats (device, n x 4, (w, x, y, z), normalised here), i.e.
 * |f^_S(R_r^T m_i)| / f^_S(0) with f^_S(k) = sum_i h^(rho_{l_i}, |k|)
 * exp(-2 pi i k . c_i / P) (Eq. (fballhat) summed directly over the knots, in
 * FP32: the band-limited spectrum of Sec. 2.5 at the turned modes, no
 * spreading).  A zero quaternion is reported by the next bc_sync as BC_ERR_ARG.
 * Asynchronous.  Errors: BC_ERR_ARG (null pointer, empty or foreign shape,
 * n < 1), BC_ERR_CUDA. */
bc_status bc_shape_moments_rot(bc_ctx_t ctx, bc_shape_t shape, const float *quats, int n, float *out);

/* Number of FP32 parameters of a network with H hidden units. */
long long bc_mlp_param_count(int hidden);

/* Creates a network on ctx's device and stream; `init` (host) holds the
 * initial parameters in the layout above.  hidden: multiple of 16 in [16, 1024].
 * Destroying the context first frees the network's device memory; the handle
 * then only accepts bc_mlp_destroy. */
bc_status bc_mlp_create(bc_ctx_t ctx, int hidden, const float *init, bc_mlp_t *out);
bc_status bc_mlp_destroy(bc_mlp_t net);

/* X (device, n x 144 floats; columns 132..143 are zero) from n device
 * quaternions (n x 4) and the two moment vectors (device).  A zero quaternion
 * is reported by the next bc_sync as BC_ERR_ARG. */
bc_status bc_mlp_features(bc_mlp_t net, const float *quats, int n, const float *moments_a, const float *moments_b,
                          float *X);

/* As bc_mlp_features with a ligand moment vector per row: moments_b_rows
 * (device, n x BC_MOMENTS), row r for rotation r (bc_shape_moments_rot). */
bc_status bc_mlp_features_rows(bc_mlp_t net, const float *quats, int n, const float *moments_a,
                               const float *moments_b_rows, float *X);

/* Which ligand moments the network takes: 0 (the default) the unrotated
 * ligand's, the same for every rotation; 1 the rotated ligand's
 * (bc_shape_moments_rot).  The learned sweeps build their features to match.
 * Errors: BC_ERR_ARG (null network, value not 0 or 1). */
bc_status bc_mlp_set_features(bc_mlp_t net, int rotated_moments);
/* The current setting (0 for a null network). */
int bc_mlp_rotated_moments(bc_mlp_t net);

/* y (device, n) = network(X). */
bc_status bc_mlp_predict(bc_mlp_t net, const float *X, int n, float *y);

/* Gradients of mean((y - t)^2) for targets t (device, n): grads (device, the
 * parameter layout; may be NULL) and loss (device, 1 float; may be NULL). */
bc_status bc_mlp_grads(bc_mlp_t net, const float *X, const float *t, int n, float *grads, float *loss);

/* One Adam step on mean((y - t)^2) with learning rate lr; loss as above. */
bc_status bc_mlp_train_step(bc_mlp_t net, const float *X, const float *t, int n, float lr, float *loss);

/* Many Adam steps in one call: `epochs` passes over the n samples (X: device,
 * n rows of the bc_mlp_features layout; t: device, n targets), each pass in a
 * pseudo-random order perm(i) = (a i + c) mod n (a coprime to n; a and c drawn
 * from splitmix64 of (seed, pass)), in floor(n / batch) batches of `batch`
 * rows gathered on the device; learning rate lr 0.5 (1 + cos(pi e / epochs))
 * in pass e.  loss (device, 1 float; may be NULL) receives the loss of the
 * last batch.  Deterministic for fixed arguments.  Asynchronous.
 * Errors: BC_ERR_ARG (null pointer, batch outside [1, n], epochs < 1,
 * lr <= 0), BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_mlp_train(bc_mlp_t net, const float *X, const float *t, int n, int batch, int epochs, float lr,
                       unsigned long long seed, float *loss);

/* Reads (get = 1) or writes (get = 0) the parameters and the two Adam moment
 * vectors (host arrays in the parameter layout; any may be NULL) and the step
 * count (may be NULL): checkpoint and resume.  Synchronous. */
bc_status bc_mlp_state(bc_mlp_t net, float *params, float *adam_m, float *adam_v, long long *step, int get);

/* Learned sweep: scores n rotations (device quats, n <= BC_TOPK_MAX) with the
 * network, keeps the topk best (ties to the lowest index), and computes the
 * peaks of their full correlations as bc_sweep does.  The features follow the
 * network's setting (bc_mlp_set_features): the unrotated ligand's moments, or
 * the rotated ligand's for every rotation.  Outputs (device):
 * idx[topk] (rotation indices, best score first), peak[topk], argmax[topk],
 * and scores[n] when not NULL.  Asynchronous.
 * Errors: BC_ERR_ARG (null pointer, n or topk out of range), BC_ERR_CUDA. */
bc_status bc_learned_sweep(bc_ctx_t ctx, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                           int topk, int *idx, float *peak, int *argmax, float *scores);

/* Learned sweep with orientation averaging: the score of rotation R is the
 * mean of the network's scores for (A, R B) and, for each of the norient host
 * quaternions s_k (w, x, y, z), for (S_k A, S_k R B), which has the same peak
 * over translations (S_k A's moments come from its spectrum, computed on the
 * device; the rotations S_k R are composed on the device, and with rotated
 * ligand moments those of S_k R B are taken).  scores, when not
 * NULL, receives the averaged scores; the rest is bc_learned_sweep, which is
 * the norient = 0 case.  Asynchronous.  Errors as bc_learned_sweep, and
 * BC_ERR_ARG for norient < 0, norient > 0 with null orients, a zero
 * orientation quaternion or an empty shape. */
bc_status bc_learned_sweep_avg(bc_ctx_t ctx, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                               int topk, const float *orients, int norient, int *idx, float *peak, int *argmax,
                               float *scores);

/* Learned sweep in two stages: the network scores all n rotations with one view
 * (the receptor as given) and keeps the best `keep`; those are scored again
 * against the receptor turned by each of the norient host orientations s_k
 * (as in bc_learned_sweep_avg), the mean of the (norient + 1) views ranks them,
 * and the topk best get full correlations as bc_sweep computes them.  The
 * turned receptor's moments come from direct sums over its knots
 * (bc_shape_moments_rot, all orientations in one launch), not from its
 * spectrum.  Outputs (device): idx[topk] (indices into quats, best first;
 * ties to the lower index), peak[topk], argmax[topk], and scores[n] (the
 * one-view scores) when not NULL.  keep = n and the same orientations rank as
 * bc_learned_sweep_avg would with those moments.  Asynchronous.  Errors:
 * BC_ERR_ARG (null pointer, n outside [1, BC_TOPK_MAX], keep outside [1, n],
 * topk outside [1, keep], norient < 0, orientations missing, a zero
 * orientation quaternion, an empty or foreign shape), BC_ERR_CUDA. */
bc_status bc_learned_sweep_cascade(bc_ctx_t ctx, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                                   int topk, const float *orients, int norient, int keep, int *idx, float *peak,
                                   int *argmax, float *scores);

/* Learned sweep with a coarse stage: the network ranks the n rotations as
 * bc_learned_sweep_cascade does (norient = 0 and keep = n: one view) and passes
 * its best `coarse_keep` on; those are correlated on the coarse context `cctx`
 * -- the same radius levels and period at a lower band limit (smaller N), with
 * Ac and Bc the shapes A and B uploaded to it -- and ranked by their coarse
 * peaks (max over cctx's translation grid, as bc_sweep computes them); the
 * topk best get full correlations on ctx.  A coarse correlation is the same
 * band-limited correlation (Eq. (ccghat)) with fewer modes: a smoother g whose
 * peak ranks rotations by their overall overlap, which the network's moments
 * rank less reliably.  Outputs (device) as bc_learned_sweep_cascade: idx[topk]
 * (indices into quats, best coarse peak first, ties to the lower index),
 * peak[topk], argmax[topk] (ctx's grid), scores[n] (one-view scores) when not
 * NULL.  cctx's stream is ordered after ctx's for the coarse stage and ctx's
 * after cctx's for the rest (events, when the streams differ).  Asynchronous.
 * Errors as bc_learned_sweep_cascade (with coarse_keep in place of topk in
 * the range checks), and BC_ERR_ARG for a null coarse context or shape, coarse
 * shapes from another context or with other knot counts than A and B, a
 * coarse context with other radius levels or period, or topk outside
 * [1, coarse_keep]. */
bc_status bc_learned_sweep_coarse(bc_ctx_t ctx, bc_mlp_t net, bc_shape_t A, bc_shape_t B, const float *quats, int n,
                                  int topk, const float *orients, int norient, int keep, bc_ctx_t cctx, bc_shape_t Ac,
                                  bc_shape_t Bc, int coarse_keep, int *idx, float *peak, int *argmax, float *scores);

/* Top-k selection: idx[0..k) (device) = indices of the k largest of scores[0..n)
 * (device), largest first, equal scores ordered by lower index.  n <= BC_TOPK_MAX.
 * Asynchronous on ctx's stream.  Errors: BC_ERR_ARG, BC_ERR_CUDA. */
bc_status bc_topk(bc_ctx_t ctx, const float *scores, int n, int k, int *idx);

/* Waits for the context stream and reports any device-side error raised by
 * earlier asynchronous calls (BC_ERR_INTERNAL, BC_ERR_TIMEOUT) or CUDA error. */
bc_status bc_sync(bc_ctx_t ctx);

/* Self-test of the bounded device-side waits: launches one thread that waits
 * on an mbarrier nothing arrives at (the wait of the tensor-core kernels), then
 * one block that waits on a work-queue counter nothing raises (the dependency
 * wait of the persistent launch).  Each wait gives up after about 2 s and
 * records its expiry in the context's error word, the kernels return, and the
 * call (which synchronises) returns BC_ERR_TIMEOUT when both expiries were
 * recorded, with the word cleared; the context stays usable.  Any other status
 * means a timeout path is broken (BC_ERR_INTERNAL when an expiry was not
 * recorded).  Errors: BC_ERR_ARG (null context), BC_ERR_OOM, BC_ERR_CUDA. */
bc_status bc_selftest_wait(bc_ctx_t ctx);

/* ---------------------------------------------------------------- profiling
 * Per-stage device times of bc_correlate, taken with CUDA events recorded on
 * the context stream between the stage launches, and the algorithmic bytes of
 * each stage (every input read once, every output written once), computed
 * from the support boxes of the last profiled call.  Stages, in launch order:
 * 0 prepare (rotation + support boxes), 1 spread, 2 fft_z, 3 fft_y,
 * 4 fft_x (with deconvolution, ball transform, level sum, conjugate product
 * and inverse x), 5 ifft_y, 6 ifft_z. */
#define BC_NUM_STAGES 7
typedef struct {
    int calls;                   /* profiled bc_correlate calls */
    long long launches;          /* kernels this library launched during them */
    double ms[BC_NUM_STAGES];    /* summed device time per stage */
    double bytes[BC_NUM_STAGES]; /* algorithmic bytes per stage and call */
} bc_profile;

/* Starts recording the next `max_calls` calls (events are created here, not in
 * the calls).  Errors: BC_ERR_ARG, BC_ERR_CUDA. */
bc_status bc_profile_begin(bc_ctx_t ctx, int max_calls);

/* Waits for the stream, fills `out` and stops recording.  Errors: BC_ERR_ARG
 * (null pointer or no bc_profile_begin), BC_ERR_CUDA. */
bc_status bc_profile_end(bc_ctx_t ctx, bc_profile *out);

/* Name of stage i (0 <= i < BC_NUM_STAGES), or "" out of range. */
const char *bc_stage_name(int i);

/* ---------------------------------------------------------------- no allocation
 * bc_correlate_noalloc: one correlation of a small pair of shapes that
 * allocates no device memory.  The paper has no counterpart; this is a
 * service for callers that cannot call cudaMalloc -- plug-ins living inside an
 * application that owns the device heap, real-time loops that must never wait
 * on the allocator.  The caller passes device buffers for the inputs and the
 * output; all other memory the computation needs is one static device array
 * of BC_NOALLOC_SCRATCH_BYTES inside this library, which every GPU that loads
 * the library keeps until the process exits.
 *
 *   params   as for bc_create, but N must be BC_NOALLOC_MAX_N (32) and
 *            level_count at most BC_NOALLOC_MAX_LEVELS (2); host memory.
 *   xyzA, levelA, nA / xyzB, levelB, nB
 *            the two shapes as in bc_shape_create, in DEVICE memory, each
 *            with at most BC_NOALLOC_MAX_KNOTS knots (0 allowed).
 *   quat     one rotation (w, x, y, z) of B, host memory.
 *   out      device buffer of N^3 floats, [kx][ky][kz]; same result as
 *            bc_correlate for one rotation (up to the rounding order of the
 *            spreading sums).
 *   cuda_stream  stream to run on (NULL = legacy default stream).
 *
 * Larger sizes are rejected with BC_ERR_ARG and a message naming the limit.
 * The call synchronises `cuda_stream` twice -- after checking the level ids
 * and coordinates, before any kernel uses them, and after the last kernel, to
 * read back the kernels' status word -- and returns with `out` complete.  A
 * status word that reports a timed-out device wait gives BC_ERR_TIMEOUT, any
 * other flag BC_ERR_INTERNAL.  The first call on a device looks up the
 * array's device address.  All calls share the one array and each call clears
 * the parts that must start at zero, so calls whose GPU work overlaps (two
 * streams, two host threads) race and corrupt each other's results.
 * Errors are reported through bc_last_error(). */
#define BC_NOALLOC_MAX_N 32
#define BC_NOALLOC_MAX_LEVELS 2
#define BC_NOALLOC_MAX_KNOTS 8192
#define BC_NOALLOC_SCRATCH_BYTES (8u << 20)
bc_status bc_correlate_noalloc(const bc_params *params, const float *xyzA, const int *levelA, int nA,
                               const float *xyzB, const int *levelB, int nB, const float *quat, float *out,
                               void *cuda_stream);

/* Message for the calling thread's most recent failure ("" if none). */
const char *bc_last_error(void);

/* Library version string. */
const char *bc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BALLCORR_H */
