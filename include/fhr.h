/*
 * fhr.h -- C ABI of libfhr, a GB300 (sm_103a) implementation of the fast
 * hyperspectral reconstruction (FHR) path of "Fast Hyperspectral Neutron
 * Tomography" (Chowdhury et al., arXiv 2410.22500), Algorithm 1:
 *
 *   counts y, open beam y0 --normalise--> p --decompose--> (V^s, D^s)
 *   --reconstruct--> x^s --expand--> x^h
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers owned by the caller, unless an entry
 *     point says otherwise.  The library never allocates device memory: calls
 *     that need scratch take a caller-provided workspace whose size is
 *     returned by the matching *_workspace_size function (256-byte aligned).
 *   - Every call is asynchronous on the stream of the context (fhr_create /
 *     fhr_set_stream).  Inputs must stay valid and outputs must not be read
 *     until the stream reaches the call.
 *   - Errors: a negative fhr_status.  Argument errors are found on the host
 *     before anything is launched; fhr_last_error() describes the last one.
 *     Errors found on the device (a bounded wait that expired, a non-finite
 *     objective) are written to a status word inside the workspace and
 *     returned by fhr_workspace_status() after a stream synchronisation.
 *     No kernel of this library traps.
 *   - Sizes are element counts; strides are in elements.
 *   - Every call makes the context's device current (cudaSetDevice) and
 *     leaves it current on return; callers that use several devices from
 *     one thread restore their own device afterwards.
 *
 * Notation (paper Sec. II): Nv views, Nr detector rows (= volume slices),
 * Nc detector columns, Nk wavelength bins, Np = Nv*Nr*Nc projections,
 * K = N_s subspace dimension, N x N image per slice.
 *
 * Layouts
 *   y   [Nv][Nr][Nc][Nk] uint16     y0 [Nr][Nc][Nk] uint16
 *   P   [Np][ldP], row j = (v*Nc + c)*Nr + r, padding columns Nk..ldP-1 zero
 *   D   [Nk][K] float (the paper's D^s)
 *   W   [Np][K] float (the paper's V^s); viewed as [Nv][Nc][Nr*K] it is the
 *       subspace sinogram, channel index w = r*K + j
 *   xs  [N][N][Nr*K] float (the paper's x^s, slice and channel innermost)
 *   xh  [Nr][N][N][Nk] float or bf16 (the paper's x^h)
 * Geometry: unit pixels centred on the origin, pixel (iy, ix) at
 * (ix - (N-1)/2, iy - (N-1)/2); unit detector bins at u_c = c - (Nc-1)/2;
 * default angles theta_v = v*pi/Nv.
 */
#ifndef FHR_H
#define FHR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fhr_status;
#define FHR_OK 0
#define FHR_ERR_ARG (-1)         /* invalid argument: null pointer, size, alignment, workspace too small */
#define FHR_ERR_CUDA (-2)        /* a CUDA runtime call failed (message in fhr_last_error) */
#define FHR_ERR_TIMEOUT (-3)     /* a device-side bounded wait expired; the kernel returned early */
#define FHR_ERR_NONFINITE (-4)   /* a non-finite value reached an objective or Gram reduction */
#define FHR_ERR_UNSUPPORTED (-5) /* parameter combination not implemented (e.g. K > 8, q != 2) */

#define FHR_F32 0
#define FHR_BF16 1

typedef struct fhr_ctx fhr_ctx;

/* Context: device ordinal and stream (a cudaStream_t, NULL = legacy default).
 * Holds only host state (device properties, last error text). */
fhr_status fhr_create(fhr_ctx **ctx, int device, void *stream);
void fhr_destroy(fhr_ctx *ctx);
fhr_status fhr_set_stream(fhr_ctx *ctx, void *stream);
const char *fhr_last_error(const fhr_ctx *ctx);
const char *fhr_version(void);

/* Launch accounting (for benchmarks; not part of Algorithm 1).  Every kernel
 * launch made through a context is counted.  fhr_profile_enable(ctx, 1)
 * resets the counters and, until disabled, brackets each launch of the timed
 * kernel families with CUDA events on the context's stream (host-side event
 * objects; no device memory).  fhr_profile_read(ctx, name, ...) synchronises
 * those events and returns the number of launches and their summed device
 * time in ms for `name` in {"normalise", "nmf_pass", "nndsvd_pass",
 * "nmf_reduce", "nmf_update", "proj_fwd", "mbir_update", "proj_bwd",
 * "expand", "fbp_filter", "mlp_forward" (a whole forward), "fmd" (a whole
 * fhr_fmd)}; with
 * name == NULL it returns the total launch count since the last enable.
 * "nmf_pass" counts the fused passes of the HALS iterations; the projection
 * passes of the NNDSVD start are counted under "nndsvd_pass". */
fhr_status fhr_profile_enable(fhr_ctx *ctx, int enable);
fhr_status fhr_profile_read(fhr_ctx *ctx, const char *name, long long *launches, double *ms);

/* Device status word kept at the start of every workspace (FHR_OK or a
 * negative code).  Synchronises the context's stream, reads it, and clears it. */
fhr_status fhr_workspace_status(fhr_ctx *ctx, void *ws);

/* ------------------------------------------------------------------------
 * Normalisation -- Eq. (neglogattenuation), p = -log(y / y0), with the
 * offset correction of Appendix A, Eq. (back_offset): when bg_mask is given,
 * b_{v,k} = mean over background pixels of -log(y/y0) and p <- p - b.
 * Readings of points the paper leaves open: counts are clamped at 1 before
 * the logarithm; p is clamped at 0 afterwards (NMF needs p >= 0); dead
 * entries give p = 0 and are left out of the background mean (a (v, k) with
 * no live background entry gets b = 0).
 *   y, y0      counts (layouts above)
 *   bg_mask    [Nr][Nc] uint8 or NULL; b_out [Nv][Nk] float receives b and
 *              is required when bg_mask is given (else may be NULL)
 *   dead_bins  uint8 or NULL: [Nk] (dead bins) or, with dead_per_pixel = 1,
 *              [Nr][Nc][Nk] (dead detector pixel-bins, the same in every view)
 *   P          output [Np][ldP], FHR_F32 (ldP % 4 == 0) or FHR_BF16 (ldP % 8 == 0)
 * ---------------------------------------------------------------------- */
typedef struct {
    int Nv, Nr, Nc, Nk;
    int ldP;              /* >= Nk */
    int p_dtype;          /* FHR_F32 or FHR_BF16 */
    int dead_per_pixel;   /* 0: dead_bins is [Nk]; 1: dead_bins is [Nr][Nc][Nk] */
} fhr_norm_params;

fhr_status fhr_normalise(fhr_ctx *ctx, const fhr_norm_params *prm,
                         const uint16_t *y, const uint16_t *y0,
                         const uint8_t *bg_mask, const uint8_t *dead_bins,
                         float *b_out, void *P);

/* ------------------------------------------------------------------------
 * Subspace decomposition -- Eq. (sub_extract_solve), min ||p - V D^T||_F^2
 * over V >= 0, D >= 0, by fast-HALS coordinate descent (Sec. III).  One
 * iteration: V half-step (Gauss-Seidel over the K coordinates of each
 * pixel), D half-step, then the columns of D are scaled to unit L2 norm
 * and V's columns by the inverse factor (the product is unchanged).  The
 * V half-step, D^T p and p V^T are one fused pass that reads P once.
 *   init  FHR_INIT_GIVEN: D, W hold the starting point on entry.
 *         FHR_INIT_NNDSVD: NNDSVD start (Sec. III) from a randomised
 *         subspace iteration for the top-K singular vectors of P, seeded
 *         by `seed` (counter-based generator, splitmix64).
 *         FHR_INIT_LEARNED (an added form, not in the paper): W0 = MLP(p_j)
 *         for every pixel (mlp, mlp_params; mlp->K == K, mlp->Nk == Nk,
 *         mlp->ldx == ldP, mlp->x_dtype == p_dtype), one pass with W0 fixed
 *         for P^T W0 and W0^T W0, then D0 from ten HALS D half-steps from
 *         D = 0; the iterations then run as from a GIVEN start.
 *         FHR_INIT_CLUSTER (the "clustering-initialised" start; the paper's
 *         Sec. III uses NNDSVD): k-means on the pixel sample
 *         j_i = floor(i Np / S), i < S = min(Np, kmeans_samples or 32768):
 *         k-means++ seeding (u_m = output m of splitmix64 from `seed`, top
 *         53 bits; centre 0 = sample floor(u_0 S), centre m = first sample
 *         whose running sum of squared distances to the nearest chosen centre
 *         exceeds u_m times their total), kmeans_iters (0: 20) Lloyd
 *         iterations (nearest centre, lowest index on ties; an empty cluster
 *         keeps its centre), all in FP64; D0 = the centres, W0 = one HALS V
 *         half-step from V = 0; the iterations then run as from GIVEN.
 *   P     [Np][ldP] in p_dtype; D [Nk][K] and W [Np][K] float, in/out.
 *   obj   device double [iters] or NULL: ||p - V D^T||^2 after each
 *         iteration, from the Gram identity in double precision.
 * K must be 1..8.  Nk <= 8192.
 * ---------------------------------------------------------------------- */
#define FHR_INIT_GIVEN 0
#define FHR_INIT_NNDSVD 1
#define FHR_INIT_LEARNED 2
#define FHR_INIT_CLUSTER 3

#define FHR_RECON_MBIR 0
#define FHR_RECON_FBP 1

struct fhr_mlp_dims_s;

typedef struct {
    int64_t Np;
    int Nk, ldP, K;
    int iters;
    int init;
    int p_dtype;
    int power_iters;   /* subspace iterations for NNDSVD (default 8 when 0) */
    uint64_t seed;
    /* FHR_INIT_LEARNED only: the warm-start network (see fhr_mlp_forward) */
    const struct fhr_mlp_dims_s *mlp;
    const float *mlp_params;
    /* FHR_INIT_CLUSTER only: pixel samples (0: 32768; at most 2^20) and
     * Lloyd iterations (0: 20) */
    int64_t kmeans_samples;
    int kmeans_iters;
} fhr_nmf_params;

fhr_status fhr_decompose_workspace_size(fhr_ctx *ctx, const fhr_nmf_params *prm, size_t *bytes);
fhr_status fhr_decompose(fhr_ctx *ctx, const fhr_nmf_params *prm, const void *P,
                         float *D, float *W, double *obj, void *ws, size_t ws_bytes);

/* Row stride of P (values per row, >= Nk) that the fused pass of fhr_decompose
 * streams fastest for rows of Nk bins in p_dtype: with it the pass copies each
 * 8-row tile of P into shared memory as one contiguous transfer instead of one
 * per row (the tile's shared-memory rows are then exactly the global rows).  The
 * extra columns must be zero, as fhr_normalise writes them.  When that stride
 * would pad a row by more than 5 % of Nk, the smallest stride fhr_normalise
 * accepts (Nk rounded up to 8 values for FHR_BF16, 4 for FHR_F32) is returned
 * instead.  Host-only: no device is touched.  Errors: FHR_ERR_ARG for Nk < 1, an
 * unknown p_dtype or a null ldP. */
fhr_status fhr_nmf_row_stride(int Nk, int p_dtype, int *ldP);

/* The same decomposition without a workspace argument, for callers that
 * cannot allocate device memory or cannot pass a workspace.  Examples: a
 * plugin bound to a fixed C signature, a framework that owns all device
 * memory through its own allocator, or a latency-critical loop where a
 * cudaMalloc (which can synchronise the device) is not allowed.  The paper has no
 * counterpart; this is a deployment form of fhr_decompose and runs its kernels.
 *   - Scratch is one static device array of 32 MiB inside the library.  Every
 *     GPU that loads the library holds it until the process exits.  Problems
 *     that need more (fhr_decompose_workspace_size) fail with FHR_ERR_ARG and
 *     a message; nothing is launched.
 *   - The call allocates nothing: no cudaMalloc, cudaFree or allocating
 *     library routine.  Event timers (fhr_profile_enable) are suspended for it.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   - All calls share the one array (it keeps the last call's contents; the
 *     call clears what must start at zero).  Calls that overlap on the GPU,
 *     from any stream or thread, race on it: serialise them.
 *   - Errors found on the device (an expired bounded wait, a non-finite
 *     objective) go to a status word kept in the array, which
 *     fhr_decompose_static_status reads; check it after the call, since the
 *     call itself returns before the device has run it.
 * Arguments as for fhr_decompose. */
fhr_status fhr_decompose_static(fhr_ctx *ctx, const fhr_nmf_params *prm, const void *P,
                                float *D, float *W, double *obj);
/* Device status of the static calls on the context's device: synchronises
 * the context's stream, returns FHR_OK or the first negative code that a
 * static call since the last read reported, and clears it.  It covers every
 * static call on the device (they share the one array), and allocates
 * nothing.  FHR_OK before the first static call on the device. */
fhr_status fhr_decompose_static_status(fhr_ctx *ctx);

/* ------------------------------------------------------------------------
 * Parallel-beam projector of Eq. (porj_matd_rel)/(recon): the strip-area
 * model A_{(v,c),i} = area(pixel i intersect strip of bin c at view v).
 * The weights are computed once per call in double precision into two
 * tables (one per direction), so the back projector is the exact transpose
 * of the forward one.  Both act on Wl values per pixel / per ray:
 *   fhr_project:     y[v][c][w] = sum_i A x[i][w]     (x [N][N][Wl], y [Nv][Nc][Wl])
 *   fhr_backproject: x[i][w]    = sum_(v,c) A y[v][c][w]
 * angles: device double [Nv] radians, or NULL for v*pi/Nv.
 * N >= 4, Nc >= 3.
 * ---------------------------------------------------------------------- */
typedef struct {
    int N, Nr, Nc, Nv;
    const double *angles;
} fhr_geom;

fhr_status fhr_projector_workspace_size(fhr_ctx *ctx, const fhr_geom *g, size_t *bytes);
fhr_status fhr_project(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *x, float *y,
                       void *ws, size_t ws_bytes);
fhr_status fhr_backproject(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *y, float *x,
                           void *ws, size_t ws_bytes);

/* ------------------------------------------------------------------------
 * MBIR of every subspace channel, Eq. (recon):
 *   x_j = argmin 1/(2 sigma_v^2) ||V_j - A x_j||^2 + beta * h(x_j),
 * h the qGGMRF prior rho(d) = |d|^p/(p sx^p) * u/(1+u), u = |d/(T sx)|^(q-p),
 * over 8 in-plane neighbours (weights 1 edge, 1/sqrt2 diagonal) and, when
 * Nr > 1, 2 inter-slice neighbours (weight 1), weights divided by their sum.
 * Solved by separable quadratic surrogates (monotone), x >= 0, optionally
 * with momentum.  All Nr slices and K channels in one pass per iteration.
 *   sino   [Nv][Nc][Nr*K] (= W from fhr_decompose)
 *   xs     [N][N][Nr*K], in: starting point, out: result
 *   sigma_v, sigma_x: host float [K] or NULL; when NULL, per channel
 *   sigma_v = rms(V_j) 10^(-snr_db/20), sigma_x = 0.2 mean(V_j) / Nc.
 * q must be 2; 1 <= p <= 2.
 * ---------------------------------------------------------------------- */
typedef struct {
    int K;
    int iters;
    float p, q, T, beta;
    float snr_db;
    int momentum;
    const float *sigma_v;
    const float *sigma_x;
} fhr_mbir_params;

fhr_status fhr_reconstruct_workspace_size(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *prm,
                                          size_t *bytes);
fhr_status fhr_reconstruct(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *prm,
                           const float *sino, float *xs, void *ws, size_t ws_bytes);

/* ------------------------------------------------------------------------
 * Filtered back-projection: the paper's faster reconstruction variant
 * ("FHR with FBP", Sec. V, Table II), in place of the MBIR of Eq. (recon).
 * Textbook parallel-beam FBP (the paper gives no discretisation): the
 * band-limited ramp filter sampled at the unit bin spacing,
 *   h[0] = 1/4, h[n] = -1/(pi n)^2 for odd n, 0 for even n != 0,
 * applied along the detector as a linear convolution (zero outside), then
 * x = (pi / Nv) A^T q with the strip-area back-projector of fhr_backproject.
 *   sino [Nv][Nc][Wl] -> xs [N][N][Wl] (Wl = Nr*K values per ray / pixel;
 *   xs 16-byte aligned when Wl % 4 == 0).  Nc <= 1024.
 * ---------------------------------------------------------------------- */
fhr_status fhr_fbp_workspace_size(fhr_ctx *ctx, const fhr_geom *geom, int Wl, size_t *bytes);
fhr_status fhr_fbp(fhr_ctx *ctx, const fhr_geom *geom, int Wl, const float *sino, float *xs,
                   void *ws, size_t ws_bytes);

/* ------------------------------------------------------------------------
 * Semi-supervised fast material decomposition (Algorithm 2 after the
 * reconstruction), from the subspace reconstruction and user regions:
 *   T[i][j] = mean of xs[n][j] over the voxels n with labels[n] == i + 1
 *             (Eq. trans_mat; labels 0 belong to no region; an empty region
 *             gives a zero row and status FHR_ERR_ARG in the workspace word),
 *   xm[n]   = argmin_{x >= 0} || xs[n] - T^T x ||^2 (Eq. mat_recon_nmf; exact
 *             Lawson-Hanson active sets in FP64, one voxel per thread),
 *   Dm      = D T^T (Eq. sub_mat_rel_basis).
 *   xs [Nx][Ns] (the [N][N][Nr*K] volume of fhr_reconstruct is [Nr*N*N][K]),
 *   labels [Nx] u8, D [Nk][Ns]; out T [Nm][Ns], xm [Nx][Nm], Dm [Nk][Nm]; all
 *   device, f32.  Ns <= 16, Nm <= min(8, Ns).  Region sums are reduced in a
 *   fixed order (deterministic).
 * ---------------------------------------------------------------------- */
fhr_status fhr_fmd_workspace_size(fhr_ctx *ctx, int64_t Nx, int Ns, int Nm, int Nk, size_t *bytes);
fhr_status fhr_fmd(fhr_ctx *ctx, int64_t Nx, int Ns, int Nm, int Nk, const float *xs, const uint8_t *labels,
                   const float *D, float *T, float *xm, float *Dm, void *ws, size_t ws_bytes);

/* ------------------------------------------------------------------------
 * Signal-to-noise ratio of a reconstruction over regions of interest
 * (Sec. V-B):
 *   FHR_SNR_FHR, Eq. (snr_fhr): 10 log10( 1/(C Nm) sum_c sum_m (mu_{m,c} / sigma_c)^2 ),
 *     x = x^h viewed as [Nx][Nk] (C = Nk): mu_{m,c} the mean of channel c over
 *     the region inside material m, sigma_c its standard deviation over the
 *     background region;
 *   FHR_SNR_FMD, Eq. (snr_fmd): 10 log10( 1/Nm sum_m (mu_m / sigma_m)^2 ),
 *     x = x^m [Nx][Nm] of fhr_fmd (C >= Nm): mu_m the mean of channel m over
 *     the region inside material m, sigma_m its deviation over the background.
 *   roi [Nx] u8: 0 = in no region, m + 1 = inside material m (m < Nm),
 *   FHR_ROI_BACKGROUND = background.  The paper's regions are 20 x 20 pixel
 *   squares; any voxel sets may be given.  sigma is the population standard
 *   deviation (over the n background voxels, divided by n).
 *   x, roi and snr_db (one double, in dB) are device pointers.  Nm <= 16,
 *   Nx < 2^31.  An empty region or background sets FHR_ERR_ARG in the
 *   workspace status word (snr_db = NaN); a zero deviation FHR_ERR_NONFINITE.
 *   Sums are FP64, in a fixed order (deterministic).
 * ---------------------------------------------------------------------- */
#define FHR_SNR_FMD 0
#define FHR_SNR_FHR 1
#define FHR_ROI_BACKGROUND 255
fhr_status fhr_snr_workspace_size(fhr_ctx *ctx, int64_t Nx, int C, int Nm, int mode, size_t *bytes);
fhr_status fhr_snr(fhr_ctx *ctx, int64_t Nx, int C, int Nm, int mode, const float *x, const uint8_t *roi,
                   double *snr_db, void *ws, size_t ws_bytes);

/* ------------------------------------------------------------------------
 * Batched MBIR: Eq. (recon) for every channel and slice of nprob independent
 * problems of uneven size in ONE persistent cooperative launch (replayed from
 * a CUDA graph), two grid-wide phases per iteration (forward residual; fused
 * backward gather + SQS update) separated by bounded grid barriers.
 * probs is a HOST array; each problem's sinogram/volume are device pointers
 * with the layouts of fhr_reconstruct (Wl = Nr*K <= 256, or <= 1024 when a
 * multiple of 4, <= 512 when even; the sinogram 16-byte
 * aligned when Wl % 4 == 0, 8-byte when Wl % 2 == 0); sigma_v[0] > 0 and
 * sigma_x[0] > 0 select explicit per-channel sigmas, else the defaults of
 * fhr_reconstruct.  All problems share the prior parameters and iteration
 * count, and must all be 2-D (Nr = 1) or all 3-D.
 * The projector tile of a work item has two dimensions:
 *   tile: rays / pixels per work item, in block-wide sweeps (0 = 2);
 *   vw:   values of a ray's / pixel's channel vector per thread (4, 2 or 1;
 *         0 = the widest that divides Nr*K), so a block sweeps 256 / (Nr*K/vw)
 *         rays or pixels at a time.  A problem whose Nr*K the requested vw does
 *         not divide takes the next smaller width that does.  Results do not
 *         depend on either (each channel is summed in the same order).
 * fhr_reconstruct_batch_autotune times every (vw, tile) pair of {4,2,1} x
 * {1,2,4,8,16} on the batch (xs is not modified; widths no problem can take
 * are skipped) and returns the fastest pair.
 * ---------------------------------------------------------------------- */
typedef struct {
    int N, Nr, Nc, Nv, K;
    const double *angles;
    const float *sino;
    float *xs;
    float sigma_v[8], sigma_x[8];
} fhr_problem;

typedef struct {
    int iters;
    float p, q, T, beta;
    float snr_db;
    int momentum;
    int tile;
    int vw;
} fhr_batch_params;

fhr_status fhr_reconstruct_batch_workspace_size(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                                const fhr_batch_params *prm, size_t *bytes);
fhr_status fhr_reconstruct_batch(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                 const fhr_batch_params *prm, void *ws, size_t ws_bytes);
fhr_status fhr_reconstruct_batch_autotune(fhr_ctx *ctx, int nprob, const fhr_problem *probs,
                                          const fhr_batch_params *prm, void *ws, size_t ws_bytes,
                                          int *best_tile, int *best_vw);

/* ------------------------------------------------------------------------
 * Subspace expansion -- Eq. (sub_expansion), x^h = x^s (D^s)^T.
 *   xs [N][N][Nr*K] float, D [Nk][K] float -> xh [Nr][N][N][Nk] in xh_dtype.
 * Bins k0..k1-1 only are written when 0 <= k0 < k1 <= Nk (a wavelength
 * slab, stored as [Nr][N][N][k1-k0]); k0 = k1 = 0 means all bins.
 * ---------------------------------------------------------------------- */
fhr_status fhr_expand(fhr_ctx *ctx, int N, int Nr, int K, int Nk, int k0, int k1,
                      const float *xs, const float *D, int xh_dtype, void *xh);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper; an added form of the decomposition's
 * start).  A 3-layer MLP maps a pixel's spectrum p (Nk bins) to K nonnegative
 * subspace coefficients:
 *   a1 = gelu(W1 p + b1), a2 = gelu(W2 a1 + b2), y = softplus(W3 a2 + b3),
 * gelu exact (erf form), softplus(z) = log(1 + e^z) (z for z > 20).
 * Parameters: one FP32 array [W1 (H1 x Nk), b1 (H1), W2 (H2 x H1), b2 (H2),
 * W3 (K x H2), b3 (K)], weights row-major [out][in].  FP32 accumulation
 * throughout; with weights_bf16 the weights and the hidden activations are
 * rounded to bf16 (round to nearest even) before each contraction.  With bf16
 * rows and bf16 weights (ldx, H1, H2 multiples of 8, X 16-byte aligned) the
 * two wide layers run on the tensor cores.
 * Inputs X: [M][ldx] rows in x_dtype (FHR_F32 or FHR_BF16), e.g. rows of P.
 * ---------------------------------------------------------------------- */
typedef struct fhr_mlp_dims_s {
    int Nk, H1, H2, K;
    int ldx;
    int x_dtype;
    int weights_bf16;
} fhr_mlp_dims;

/* Workspace for fhr_mlp_forward (train = 0) or fhr_mlp_grad (train = 1). */
fhr_status fhr_mlp_workspace_size(fhr_ctx *ctx, const fhr_mlp_dims *dims, int train, size_t *bytes);
/* Y [M][K] float = MLP(X) for any M (processed in chunks of 65536 rows). */
fhr_status fhr_mlp_forward(fhr_ctx *ctx, const fhr_mlp_dims *dims, const float *params, int64_t M,
                           const void *X, float *Y, void *ws, size_t ws_bytes);
/* Mean-squared error against T [M][K] (loss, a device double, may be NULL)
 * and its gradient with respect to every parameter (grad: same layout as
 * params, overwritten).  1 <= M <= 32768 rows per call. */
fhr_status fhr_mlp_grad(fhr_ctx *ctx, const fhr_mlp_dims *dims, const float *params, int64_t M,
                        const void *X, const float *T, float *grad, double *loss, void *ws, size_t ws_bytes);
/* One AdamW step (decoupled weight decay) on n parameters, step >= 1:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr ((m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps) + weight_decay w). */
fhr_status fhr_mlp_adamw(fhr_ctx *ctx, int64_t n, float *params, const float *grad, float *m, float *v,
                         int step, float lr, float beta1, float beta2, float eps, float weight_decay);

/* ------------------------------------------------------------------------
 * Algorithm 1 end to end: normalise -> decompose -> reconstruct -> expand.
 * With host_io = 0, y, y0 and xh are device pointers.  With host_io = 1 they
 * are HOST pointers: the counts are copied in and x^h copied out through
 * staging buffers in the workspace, with asynchronous copies on the
 * context's stream (pinned host memory makes them truly asynchronous).
 * bg_mask, dead_bins are device pointers or NULL.  D_out [Nk][K] device
 * float, obj device double [nmf.iters] or NULL.  nmf.init is
 * FHR_INIT_NNDSVD, FHR_INIT_CLUSTER or FHR_INIT_LEARNED (nmf.mlp with
 * ldx = norm.ldP and x_dtype = norm.p_dtype); FHR_INIT_GIVEN is rejected, the
 * pipeline having no starting point of its own.  The reconstruction starts
 * from x^s = 0.  Sizes in norm, nmf, geom and mbir
 * must agree (Np = Nv*Nr*Nc, geom.Nr = norm.Nr, mbir.K = nmf.K).
 * ---------------------------------------------------------------------- */
typedef struct {
    fhr_norm_params norm;
    fhr_nmf_params nmf;
    fhr_geom geom;
    fhr_mbir_params mbir;
    int xh_dtype;
    int host_io;
    int recon;   /* FHR_RECON_MBIR (Eq. recon, default) or FHR_RECON_FBP (fhr_fbp) */
} fhr_pipeline_params;

/* With host_io, y and y0 are pinned host buffers copied in on a copy stream
 * and xh a pinned host buffer copied out on another: the call returns with the
 * output copy pending, and consecutive calls overlap their copies with each
 * other's compute.  The host buffers must stay untouched until the copies
 * are done: fhr_io_join orders the context stream after the last output copy,
 * and fhr_workspace_status waits for it (as does a device synchronisation). */
fhr_status fhr_io_join(fhr_ctx *ctx);
fhr_status fhr_pipeline_workspace_size(fhr_ctx *ctx, const fhr_pipeline_params *prm, size_t *bytes);
fhr_status fhr_pipeline(fhr_ctx *ctx, const fhr_pipeline_params *prm,
                        const uint16_t *y, const uint16_t *y0,
                        const uint8_t *bg_mask, const uint8_t *dead_bins,
                        float *D_out, void *xh, double *obj, void *ws, size_t ws_bytes);

#ifdef __cplusplus
}
#endif
#endif /* FHR_H */
