/*
 * ttm.h -- C ABI of libttm: tensorial template matching (TTM) on one GB300
 * GPU (sm_103a), after Martinez-Sanchez, Homberg, Almira & Phelippeau,
 * "Tensorial template matching for fast cross-correlation with rotations and
 * its application for tomography" (ECCV 2024).
 *
 * Conventions (all entry points):
 *   - Volumes are C-order float32 arrays [Z][Y][X], x fastest. A template of
 *     extent (tz,ty,tx) has its centre at (tz/2, ty/2, tx/2); offsets are
 *     p = (ix-cx, iy-cy, iz-cz) and vectors are ordered (x, y, z).
 *   - A symmetric tensor of degree n over R^3 is stored by its K =
 *     binom(n+2, 2) independent components (the full-tensor entries), in
 *     graded-lex descending order of the exponents (a,b,c) of (x,y,z): for
 *     n = 2 that is xx, xy, xz, yy, yz, zz. Multi-component fields are
 *     structure-of-arrays [K][...].
 *   - Quaternions are (w, x, y, z); rotation R(q) acts on column vectors and
 *     a rotated template is t_R(p) = t(R^T p) (trilinear, zero outside).
 *   - Pointers named d_* are device pointers, h_* host pointers. All buffers
 *     are owned by the caller; the library allocates only in *_create calls
 *     (context workspace, plans) and never inside the compute calls.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Compute calls
 *     are asynchronous on it unless stated otherwise.
 *   - Every call returns a ttm_status; TTM_OK is 0. On failure nothing has
 *     been written to the outputs except where stated, and a message is kept
 *     in the context (ttm_last_error). No C++ exception crosses this ABI.
 *   - Results are defined on the valid interior: voxels whose whole template
 *     window lies inside the volume. Outside it values are finite but
 *     implementation defined (the correlation wraps around the grid there).
 */
#ifndef TTM_H
#define TTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TTM_OK = 0,
    TTM_E_INVALID_ARG = 1, /* null pointer, bad enum, bad parameter */
    TTM_E_SHAPE = 2,       /* volume smaller than the template, or size not supported */
    TTM_E_UNSUPPORTED = 3, /* order n / d' / precision not built */
    TTM_E_OOM = 4,         /* device allocation failed in a *_create call */
    TTM_E_CUDA = 5,        /* a CUDA runtime call failed (message in ttm_last_error) */
    TTM_E_TIMEOUT = 6,     /* a bounded device wait expired (ttm_ctx_device_status) */
    TTM_E_INTERNAL = 7
} ttm_status;

typedef enum {
    TTM_PREC_FP32 = 0,         /* template spectra stored and multiplied in FP32 */
    TTM_PREC_FP16_SPECTRA = 1, /* spectra in FP16 with a per-component scale, FP32 accumulate */
    TTM_PREC_BF16_SPECTRA = 2  /* spectra in BF16 with a per-component scale, FP32 accumulate */
} ttm_precision;

typedef enum {
    TTM_MAX_PLAIN = 0,   /* probe directions + Newton polish */
    TTM_MAX_MLP_WARM = 1 /* learned warm start, plain maximiser as fallback */
} ttm_maximiser;

typedef struct ttm_ctx ttm_ctx;
typedef struct ttm_plan ttm_plan;
typedef struct ttm_mlp ttm_mlp;

/* Parameters of the tensor field and of the local normalisation.
 *   order_n          tensor degree n (even; 2, 4 or 6 are built)
 *   dprime           3: the weight of rotation R is (R e_z)^{(x)n}, maximised
 *                    over unit directions u in S^2 (K = binom(n+2,2));
 *                    4: the quaternion powers q^{(x)n} of Sec. 3, maximised
 *                    over unit quaternions (K = binom(n+3,3): 10, 35, 84):
 *                    a full rotation, roll included. Field, correlation
 *                    and maximiser are built for n = 2, 4, 6; the learned
 *                    maximiser and the batch are d' = 3 only
 *   mask_radius      r of the spherical mask m (Sec. 2, after Eq. 3), voxels
 *   mask_soft_width  width of the raised-cosine edge beyond r; 0 = binary
 *   filter_a         a of the filter h with z-transform 1 + a(z + 1/z - 2)
 *                    (Sec. 2; the paper uses 1/5); 0 disables the filter
 *   n_rot_base       super-Fibonacci samples of SO(3) for Eq. 9
 *   cube_symmetrize  1: the quadrature is the 24 cube rotations times the
 *                    base samples (24 * n_rot_base rotations)            */
typedef struct {
    int order_n;
    int dprime;
    double mask_radius;
    double mask_soft_width;
    double filter_a;
    int64_t n_rot_base;
    int cube_symmetrize;
} ttm_field_params;

/* Fills p with the defaults: n = 4, d' = 3, r = 16, soft 0, a = 0.2,
 * 2048 base rotations, cube symmetrisation on. */
void ttm_default_params(ttm_field_params* p);

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device` (makes it current). */
ttm_status ttm_ctx_create(int device, ttm_ctx** out);
void ttm_ctx_destroy(ttm_ctx* ctx);
/* Text of the last failure on this context ("" if none). Owned by ctx. */
const char* ttm_last_error(const ttm_ctx* ctx);
/* Bounded device waits (no paper counterpart; failure detection). Kernels
 * of this library that wait on asynchronous copies (the TMA-staged fused z
 * pass of ttm_correlate, tm_correlate and the batch) poll each wait at most
 * `polls` times (default 4194304, far beyond a copy's microseconds). When a
 * wait expires the kernel records it in the context, waits with a fixed
 * limit for its own copies in flight and returns without writing its
 * output; the context stays usable.
 *   ttm_ctx_set_wait_limit: sets the poll limit (>= 0; 0 makes every such
 *     wait expire at once, which exercises the error path).
 *   ttm_ctx_device_status: synchronises `stream` and returns TTM_E_TIMEOUT
 *     if a bounded wait of this context expired since the last check (the
 *     outputs of the calls in between are undefined), else TTM_OK; clears
 *     the record. */
ttm_status ttm_ctx_set_wait_limit(ttm_ctx* ctx, int64_t polls);
ttm_status ttm_ctx_device_status(ttm_ctx* ctx, void* stream);
/* binom(n + d' - 1, n): the number of independent components (Sec. 3). */
int ttm_num_components(int order_n, int dprime);
/* Library version string, e.g. "ttm 0.1 sm_103a". */
const char* ttm_version(void);

/* The rotation quadrature of Eq. 9 (host only, no device work): n_base
 * super-Fibonacci unit quaternions (Alexa, CVPR 2022; the sampling the paper
 * uses in Sec. 3 and Sec. 3.4), optionally left-multiplied by the 24 cube
 * rotations (entry i*24 + j = c_j * q_i). h_quats receives 4 * count
 * doubles where count = n_base * (cube ? 24 : 1). */
ttm_status ttm_rotation_set(int64_t n_base, int cube, double* h_quats);

/* ----------------------------------------------------- step a0: Alg. 1 */

/* Tensor template (Eq. 9, Alg. 1): normalises the template (Eq. 4: filter
 * h, mask m, zero mean and unit norm under the mask) into t', then
 * T_alpha(p) = (1/|Q|) sum_q u_q^alpha t'(R_q^T p) over the quadrature of
 * `params` (u_q = R_q e_z for d' = 3, u_q = q for d' = 4), all in FP64 on
 * the GPU. Components are in graded-lex descending order of the exponents
 * of (x, y, z), or of (w, x, y, z) for d' = 4.
 *   d_tmpl   float32 [tz][ty][tx] raw template (device)
 *   d_field  float64 [K][tz][ty][tx] output (device), K = ttm_num_components
 * Blocking: returns once the field has been written. */
ttm_status ttm_build_tensor_field(ttm_ctx* ctx, const float* d_tmpl, int tz, int ty, int tx,
                                  const ttm_field_params* params, double* d_field, void* stream);

/* -------------------------------------------------- steps a1-a2: Alg. 2 */

/* A plan binds a tensor field to one tomogram shape: it holds the template
 * spectra (transformed along x and y, kept on the template's z rows), the
 * spectrum of the mask, and the per-tomogram workspace. Allocates device
 * memory (~ (K + 6) * Z*Y*(X/2+1) * 8 bytes for FP32). Blocking; the first
 * plan of a context with a new extent also times the double-float
 * transform kernels for it (a few milliseconds, kept in the context).
 *   precision  TTM_PREC_FP32, or TTM_PREC_FP16_SPECTRA / _BF16_SPECTRA:
 *              the template spectra and the K-component work buffer are
 *              stored as 16-bit pairs (half the bytes), each component
 *              scaled by 1 / max |its partial spectrum|, the image spectrum
 *              divided by its largest modulus, and the z- and y-pass stores
 *              scaled by fixed factors that keep the a-priori bounds
 *              (Z tz, then Z tz Y) below 2^15; all transform arithmetic and
 *              the output C stay FP32, the local variance FP64. Expected
 *              error of C: about one unit roundoff (2^-11 FP16, 2^-8 BF16)
 *              relative, at most three. */
ttm_status ttm_plan_create(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                           const ttm_field_params* params, int Z, int Y, int X,
                           ttm_precision precision, ttm_plan** out);

/* As ttm_plan_create, for a Zt x Yt x Xt tomogram correlated on a larger
 * Z x Y x X working grid (zero padded; each working extent >= the
 * tomogram's). The FFT lengths are the working extents, so a tomogram of
 * any size can use lengths with fast transforms (ttm_autotune_shape picks
 * them). Within the valid box (ttm_plan_valid_box, tomogram coordinates,
 * which are also working-grid coordinates) the results equal those of an
 * unpadded plan: no template offset leaves the tomogram there. Every map
 * (d_C, d_score, ...) is laid out on the working grid; d_tomo passed to
 * ttm_correlate is the Zt x Yt x Xt tomogram. */
ttm_status ttm_plan_create_padded(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                                  const ttm_field_params* params, int Zt, int Yt, int Xt, int Z,
                                  int Y, int X, ttm_precision precision, ttm_plan** out);
void ttm_plan_destroy(ttm_plan* plan);
/* Number of components K of the plan. */
int ttm_plan_components(const ttm_plan* plan);
/* Valid-interior box of the plan: z0,z1,y0,y1,x0,x1 (half-open). */
void ttm_plan_valid_box(const ttm_plan* plan, int* box6);

/* Tensorial correlation C_alpha(x) = w(x) (g * T_alpha)(x) (Eq. 8, Alg. 2)
 * with g = h * f (Eq. 3, zero padded), the correlation of Eq. 5 evaluated
 * through FFTs (periodic on the Z x Y x X grid), and the local normaliser
 * of Eq. 2: w = 1/sqrt(S2 - S1^2/M), S1 = sum m g(x+.), S2 = sum m^2
 * g(x+.)^2, summed in FP64; w = 0 where the local variance is zero to
 * rounding: at most 1e-8 * M * mean(g^2) (a window too empty for the FP32
 * correlation to resolve) or at most 1e-10 * S2.
 *   d_tomo  float32 [Z][Y][X] (device)
 *   d_C     float32 [K][Z][Y][X] output (device) */
ttm_status ttm_correlate(ttm_plan* plan, const float* d_tomo, float* d_C, void* stream);

/* Arithmetic of the local sums S1, S2 and of the variance of Eq. 2:
 *   TTM_LOCALSUM_FP64 (default): FP64 transforms and FP64 variance;
 *   TTM_LOCALSUM_DF64: double-float arithmetic (each value an unevaluated
 *   sum of two FP32 numbers, ~48-bit significand, FP32 exponent range) on the
 *   FP32 pipes, variance formed in double-float.
 * Takes effect at the next ttm_correlate. */
typedef enum { TTM_LOCALSUM_FP64 = 0, TTM_LOCALSUM_DF64 = 1 } ttm_localsum_precision;
ttm_status ttm_plan_set_localsum(ttm_plan* plan, int mode);

/* Local normaliser w of the last ttm_correlate on this plan, float32
 * [Z][Y][X] copied to d_w (device). */
ttm_status ttm_plan_copy_w(ttm_plan* plan, float* d_w, void* stream);

/* ---------------------------------------------------- steps a3-a4: Sec. 3.1-3.2 */

/* Per voxel: score s(x) = max over unit u of C(x) . u^{(x)n} (the dominant
 * Z-eigenvalue, Sec. 3.1), orientation u*(x) (the maximiser) and the
 * Frobenius proxy ||C(x)||_F (Sec. 3.2).
 *   d_C       float32 [K][Z][Y][X] (device, from ttm_correlate)
 *   d_score   float32 [Z][Y][X]
 *   d_orient  float32 [d'][Z][Y][X]: d' = 3, the unit direction (u_x, u_y,
 *             u_z) with its last non-zero coordinate positive; d' = 4, the
 *             unit quaternion (w, x, y, z) with its first non-zero entry
 *             positive (q and -q are the same rotation)
 *   d_frob    float32 [Z][Y][X] or NULL
 *   mode      TTM_MAX_PLAIN: probe directions (tensor-core probe product),
 *             angularly separated starts, Newton polish;
 *             TTM_MAX_MLP_WARM (d' = 3): the MLP's direction (BF16 tensor
 *             cores) is polished by Newton and kept where the polish
 *             converged, its value is not below the best of the 128 probe
 *             directions (up to their FP16 error bound), the plain
 *             maximiser would take one start only and the direction lies
 *             within 20 degrees of the best probe; the other voxels go
 *             through the plain maximiser (their count is read with
 *             ttm_plan_fallback_count). The paper maximises with SS-HOPM
 *             (Sec. 3.1); the learned start has no counterpart there.
 *   mlp       NULL for TTM_MAX_PLAIN; for TTM_MAX_MLP_WARM an MLP with
 *             K inputs on the plan's device. The first call after the MLP's
 *             parameters change rebuilds its BF16 image (synchronous).
 * The learned mode uses the plan's peak-candidate scratch for its fallback
 * list: calls on one plan must not overlap. */
ttm_status ttm_peak_map(ttm_plan* plan, const float* d_C, ttm_maximiser mode, const ttm_mlp* mlp,
                        float* d_score, float* d_orient, float* d_frob, void* stream);

/* Voxels the last TTM_MAX_MLP_WARM ttm_peak_map on this plan handed to the
 * plain maximiser. Synchronises `stream`. */
ttm_status ttm_plan_fallback_count(ttm_plan* plan, int64_t* h_count, void* stream);

/* ------------------------------------------- learned warm start (no paper
 * counterpart): an MLP K -> 128 -> 128 -> 3 with GELU (tanh form) and the
 * output normalised to a unit vector, trained to predict the maximiser u*
 * of C . u^{(x)n} from x = C / ||C||_F, loss 1 - (u_hat . u*)^2 (the same
 * for u* and -u*, as the even form is).
 * Parameters are one flat FP32 array: W1 [128][K], b1 [128], W2 [128][128],
 * b2 [128], W3 [3][128], b3 [3] (ttm_mlp_num_params(K) floats). */

/* Number of parameters of the MLP with K inputs (0 if K <= 0). */
int64_t ttm_mlp_num_params(int n_inputs);
/* Creates an MLP with n_inputs (1..128) inputs on ctx's device: weights
 * N(0, 1/fan_in) from a SplitMix64 stream of `seed`, biases 0; Adam state 0.
 * Allocates parameters, gradients, Adam moments (blocking). */
ttm_status ttm_mlp_create(ttm_ctx* ctx, int n_inputs, uint64_t seed, ttm_mlp** out);
void ttm_mlp_destroy(ttm_mlp* mlp);
int ttm_mlp_inputs(const ttm_mlp* mlp);
/* Host copy of the parameters (ttm_mlp_num_params floats), blocking. */
ttm_status ttm_mlp_get_params(const ttm_mlp* mlp, float* h_params);
/* Sets the parameters from host memory and resets the Adam state. */
ttm_status ttm_mlp_set_params(ttm_mlp* mlp, const float* h_params);
/* FP32 forward: d_U [n][3] = u_hat of the rows of d_X [n][K] (device).
 * Grows the MLP's training scratch on first use (allocates). */
ttm_status ttm_mlp_forward(ttm_mlp* mlp, const float* d_X, int64_t n, float* d_U, void* stream);
/* FP32 loss sum over the n rows and its gradient (d_grad, num_params
 * floats, device) with targets d_U [n][3]; *h_loss on the host
 * (synchronises). Grows the training scratch on first use. */
ttm_status ttm_mlp_loss_grad(ttm_mlp* mlp, const float* d_X, const float* d_U, int64_t n,
                             float* d_grad, double* h_loss, void* stream);
/* Adam (beta 0.9 / 0.999, eps 1e-8) on the mean loss of minibatches of
 * `batch` rows, `epochs` passes over a SplitMix64 permutation of the n
 * pairs per epoch (seeded); whole batches only. *h_last_loss = mean loss of
 * the last batch of the last epoch. Blocking; allocates its permutation. */
ttm_status ttm_mlp_train(ttm_mlp* mlp, const float* d_X, const float* d_U, int64_t n, int epochs,
                         int batch, float lr, uint64_t seed, double* h_last_loss, void* stream);
/* Arithmetic of the forward and backward products of ttm_mlp_forward,
 * ttm_mlp_loss_grad and ttm_mlp_train:
 *   TTM_MLP_FP32 (default): FP32 operands and accumulation (the mode whose
 *     gradient is checked against an FP64 reference);
 *   TTM_MLP_BF16: operands rounded to BF16 and multiplied on the tensor
 *     cores with FP32 accumulation (mixed-precision training); parameters,
 *     gradients, activations between layers and the Adam state stay FP32. */
typedef enum { TTM_MLP_FP32 = 0, TTM_MLP_BF16 = 1 } ttm_mlp_precision;
ttm_status ttm_mlp_set_precision(ttm_mlp* mlp, int mode);
/* BF16 tensor-core inference (the arithmetic of the learned maximiser):
 * d_U [n][3] from d_X [n][K]; K <= 32. */
ttm_status ttm_mlp_infer(ttm_mlp* mlp, const float* d_X, int64_t n, float* d_U, void* stream);
/* Training pairs from maps: for each linear voxel index d_idx[i] (device
 * int64, < V), d_X[i] = C(v) / ||C(v)||_F (zeros where the norm is 0) and
 * d_U[i] = d_orient(v); C float32 [K][V] of order order_n (d' = 3). */
ttm_status ttm_mlp_make_pairs(ttm_ctx* ctx, const float* d_C, int order_n, int64_t V,
                              const float* d_orient, const int64_t* d_idx, int64_t n, float* d_X,
                              float* d_U, void* stream);
/* File: 8-byte magic "TTMMLP1", int32 K, int32 128, int64 num_params,
 * float32 parameters (host byte order). */
ttm_status ttm_mlp_save(const ttm_mlp* mlp, const char* path);
ttm_status ttm_mlp_load(ttm_ctx* ctx, const char* path, ttm_mlp** out);

/* --------------------------------------------------------- step a5: Sec. 3.4 */

/* Find Peaks: the P highest local maxima (26-neighbourhood, within the valid
 * box; ties broken by lower linear index) of d_map [Z][Y][X] that keep a
 * Euclidean distance >= min_dist (the paper: 2 x mask radius) to every
 * higher accepted peak. Writes up to P linear indices and values to host
 * arrays and the count to *h_count. Synchronises `stream`. */
ttm_status ttm_find_peaks(ttm_plan* plan, const float* d_map, int P, double min_dist,
                          int64_t* h_idx, float* h_val, int* h_count, void* stream);

/* Allocation-free Find Peaks. The paper has no counterpart to this entry
 * point: it returns exactly what ttm_find_peaks returns for the same map,
 * box, P and min_dist, but allocates no memory, device or library, and needs
 * no plan. It serves callers that cannot allocate device memory where they
 * need peaks: a process whose free device memory is reserved by another
 * allocator (a framework's caching pool), or a streaming loop in which
 * cudaMalloc / cudaFree would synchronise the device and stall the work on
 * other streams.
 *   d_map    float32 [Z][Y][X] (device); every extent below 2^21
 *   box      host int[6]: z0, z1, y0, y1, x0, x1 (half-open), the search
 *            region (ttm_plan_valid_box gives the valid box of a plan)
 *   h_idx, h_val, h_count: as ttm_find_peaks (host; room for P entries)
 * Scratch is one fixed device array inside the library (about 3.3 MB per
 * device): at most 262144 local maxima in the box and P <= 16384. A larger
 * P, or a map with more local maxima in the box, fails with TTM_E_SHAPE
 * (nothing written to h_idx / h_val). The set-up is done by ttm_ctx_create:
 * it looks up the device address of that array with the context's device
 * current, which (under CUDA's lazy module loading) is also when the
 * array's device memory is committed on that device; this call does no
 * set-up of its own. The selection takes at most P passes over the
 * surviving candidates on one SM (about 0.2 ms per pass over 262144).
 * Every call clears the array's candidate counter on `stream` before use.
 * All calls on one device share the array: calls that overlap (on other
 * streams or host threads) race and must be serialised by the caller.
 * Synchronises `stream`. */
ttm_status ttm_find_peaks_noalloc(ttm_ctx* ctx, const float* d_map, int Z, int Y, int X,
                                  const int* box, int P, double min_dist, int64_t* h_idx,
                                  float* h_val, int* h_count, void* stream);

/* Position refinement, TTM-ref (Sec. 3.3, Alg. 3). For each peak x_i the
 * voxels x of the ball ||x - x_i|| <= r_s (x_i first, then the rest in
 * z, y, x order) inside the valid box are scored by the LNCC at their own
 * optimal rotation, c(x) = w(x) sum_z t'(R(q*(x))^T z) g(x + z), evaluated
 * in real space over the template window (trilinear samples of t', FP32
 * samples, FP64 reduction); the first strictly highest voxel in that order
 * is kept (the paper uses r_s = 3).
 *   plan      a d' = 4 plan after ttm_correlate: g and w of that call are used
 *   d_tmpl    float32 [tz][ty][tx] raw template (device); normalised here by
 *             Eq. 4 with the plan's parameters, as in ttm_build_tensor_field
 *   d_orient  float32 [4][Z][Y][X] quaternion map of ttm_peak_map (device)
 *   h_peaks   int64 [P] linear voxel indices on the plan's working grid,
 *             each inside the valid box (host); P <= 65535
 *   h_idx     int64 [P] refined voxel indices; h_quat float32 [P][4] its
 *             rotation (w, x, y, z); h_lncc float32 [P] its LNCC (host)
 * Allocates a small per-call workspace; synchronises `stream`. Errors:
 * TTM_E_UNSUPPORTED for a d' = 3 plan, TTM_E_INVALID_ARG for a peak outside
 * the valid box or r_s outside [0, 16]. */
ttm_status ttm_refine_peaks(ttm_plan* plan, const float* d_tmpl, const float* d_orient, const int64_t* h_peaks,
                            int P, double r_s, int64_t* h_idx, float* h_quat, float* h_lncc, void* stream);

/* ------------------------------------- block processing: Sec. 3.4 */

/* The z-slab partition of block processing (host only). For a tomogram of
 * Z planes and a template of tz planes (centre cz = tz / 2; valid planes
 * [cz, Z - (tz - cz) + 1)), slab k gets the output planes [o0, o1) (slab_z
 * of the valid planes, the last one ragged), its map planes [m0, m1) =
 * [o0, o1) widened by one valid plane each side (the 26-neighbour test), and
 * its input planes [i0, i1) = the map planes' template windows plus one
 * plane each side for the 3-tap filter, clipped to the tomogram. Writes up
 * to cap rows (o0, o1, m0, m1, i0, i1) to out (may be NULL) and returns the
 * slab count, or -1 for bad arguments. */
int ttm_slab_ranges(int Z, int tz, int slab_z, int* out, int cap);

/* Merge Peaks (Sec. 3.4, host only): orders n candidates (linear indices
 * on a Z x Y x X grid, values) by value descending then index ascending and
 * accepts greedily those at Euclidean distance >= min_dist from every one
 * accepted before, up to P. Returns the count written to out_idx / out_val,
 * or -1 for bad arguments. Find Peaks is this applied to the strict
 * 26-neighbour maxima of a map. */
int ttm_merge_peaks(int64_t n, const int64_t* idx, const float* val, int Z, int Y, int X, int P, double min_dist,
                    int64_t* out_idx, float* out_val);

/* Block processing (Sec. 3.4): Find Peaks of the score map (map_kind 0) or
 * of the Frobenius map (map_kind 1) of a tomogram held in HOST memory,
 * float32 [Z][Y][X], processed in z-slabs of slab_z output planes
 * (ttm_slab_ranges). Each slab is copied to the device, correlated on its
 * own autotuned working grid (one plan per slab depth, FP32, FP64 local
 * sums) and scored by the plain maximiser; the strict 26-neighbour maxima
 * of its output planes are merged over all slabs (ttm_merge_peaks). The
 * candidates and their order are those of ttm_find_peaks on the whole
 * tomogram. The one difference is that the variance floor of Eq. 2
 * (reading of zero variance) uses each slab's mean of g^2. The values
 * differ by the rounding of the different FFT lengths.
 *   d_field   float64 [K][tz][ty][tx] (device), params as for ttm_plan_create
 *   h_idx, h_val  P entries (host): tomogram linear indices and map values
 * One call: ttm_blocked_create, ttm_blocked_run, ttm_blocked_destroy
 * (allocates the slab workspace for the call); synchronises `stream`. */
ttm_status ttm_blocked_peaks(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                             const ttm_field_params* params, const float* h_tomo, int Z, int Y, int X, int slab_z,
                             int map_kind, int P, double min_dist, int64_t* h_idx, float* h_val, int* h_count,
                             void* stream);

/* The same block processing as a session kept across tomograms of one
 * shape (no paper counterpart: an execution scheme). ttm_blocked_create
 * computes the slab table, one plan per distinct slab depth (the template
 * spectra on each slab's working grid) and the slab buffers; allocates,
 * blocking. ttm_blocked_run processes one Z x Y x X host tomogram: slab
 * k + 1 is uploaded on the session's own copy stream while the kernels of
 * slab k run on `stream` (the copies overlap the kernels when h_tomo is
 * pinned host memory), the candidates of all slabs are gathered on the
 * device and read back once, then merged (ttm_merge_peaks); synchronises
 * `stream`. Runs of one session must not overlap. */
typedef struct ttm_blocked ttm_blocked;
ttm_status ttm_blocked_create(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                              const ttm_field_params* params, int Z, int Y, int X, int slab_z, ttm_blocked** out);
ttm_status ttm_blocked_run(ttm_blocked* session, const float* h_tomo, int map_kind, int P, double min_dist,
                           int64_t* h_idx, float* h_val, int* h_count, void* stream);
void ttm_blocked_destroy(ttm_blocked* session);

/* ------------------------------------------------------- step a6: Eqs. 1, 6, 7 */

/* Classical template matching baseline: for every rotation q_j of h_quats
 * (4 * n_rot doubles, any order), c(x, R_j) = w(x) (g * t'_{R_j})(x) with
 * t' of Eq. 4; d_best[x] = max_j c, d_best_idx[x] = the first j attaining
 * it. Uses the same filter, mask and normaliser as ttm_correlate.
 *   d_tomo float32 [Z][Y][X]; d_tmpl float32 [tz][ty][tx] raw template
 *   d_best float32 [Z][Y][X]; d_best_idx int32 [Z][Y][X] (device)
 * Allocates its workspace for the duration of the call (blocking). */
ttm_status tm_correlate(ttm_ctx* ctx, const float* d_tomo, int Z, int Y, int X, const float* d_tmpl,
                        int tz, int ty, int tx, const ttm_field_params* params,
                        const double* h_quats, int64_t n_rot, float* d_best, int32_t* d_best_idx,
                        void* stream);

/* ------------------------------------------ batched TTM and FFT autotuner
 * (no paper counterpart: an execution scheme for many tomograms) */

/* Autotuner: for each FP32 transform length it times the register kernel
 * (where one exists) and the shared-memory passes over radix schedules and
 * tile widths, and keeps the fastest in the context; plans and batches
 * created afterwards use the tuned schedules. ttm_autotune_shape picks the
 * working grid (each extent a 7-smooth length in [n, 1.34 n]) of a
 * Z x Y x X tomogram that minimises the modelled transform time, tuning the
 * lengths it needs (timed on the device: allocates a scratch buffer and
 * synchronises). zyx receives 3 ints. */
ttm_status ttm_autotune_shape(ttm_ctx* ctx, int Z, int Y, int X, int* zyx);
/* Number of tuned lengths held by the context. */
int ttm_autotune_entries(const ttm_ctx* ctx);
/* Tuned records as JSON (one object per line: L, kind (0 FP32, 2 double-
 * float), reg, W, rad, us_line); double-float lengths are tuned (register
 * against shared-memory pass) on their first use by a plan of the context;
 * load replaces records of the same length and rejects malformed files
 * with TTM_E_INVALID_ARG. */
ttm_status ttm_autotune_save(const ttm_ctx* ctx, const char* path);
ttm_status ttm_autotune_load(ttm_ctx* ctx, const char* path);

typedef struct ttm_batch ttm_batch;
typedef struct {
    const float* d_tomo; /* float32 [Z][Y][X] (device); read at every ttm_batch_run */
    int Z, Y, X;
} ttm_batch_tomo;
typedef struct {
    int tomo;        /* index into the tomogram list */
    int tmpl;        /* index into the field list */
    float* d_score;  /* float32 [Z][Y][X] of the tomogram (device) */
    float* d_orient; /* float32 [3][Z][Y][X] */
    float* d_frob;   /* float32 [Z][Y][X] or NULL */
} ttm_batch_item;
enum { TTM_BATCH_AUTOTUNE = 1, TTM_BATCH_LOCALSUM_DF64 = 2 };

/* Batched TTM over (tomogram, template) pairs: all tomograms share
 * `params` and the template shape tz x ty x tx; d_fields[j] is the
 * K x tz x ty x tx FP64 field of template j (ttm_build_tensor_field).
 * Each tomogram is correlated on a zero-padded working grid
 * (TTM_BATCH_AUTOTUNE: ttm_autotune_shape, else the next 7-smooth extents)
 * with one preparation shared by its pairs; each pair writes the plain
 * maximiser's score, orientation (and Frobenius norm) inside its valid box
 * (tomogram coordinates; other voxels are not written). The pairs run on
 * n_branches (1..16) concurrent paths, balanced by modelled cost, and the
 * whole batch is captured once into a CUDA graph. Allocates the
 * preparations, the spectra of every pair and one work and C buffer per
 * branch; blocking. TTM_BATCH_LOCALSUM_DF64 selects the double-float local
 * sums (ttm_plan_set_localsum). */
ttm_status ttm_batch_create(ttm_ctx* ctx, const ttm_field_params* params, int tz, int ty, int tx,
                            int n_templates, const double* const* d_fields, int n_tomos,
                            const ttm_batch_tomo* tomos, int n_items, const ttm_batch_item* items,
                            int n_branches, int flags, ttm_batch** out);
/* One launch of the batch's graph on `stream` (asynchronous). Calls on one
 * batch must not overlap. */
ttm_status ttm_batch_run(ttm_batch* batch, void* stream);
/* Working grid chosen for tomogram `tomo` (3 ints). */
ttm_status ttm_batch_work_shape(const ttm_batch* batch, int tomo, int* zyx);
void ttm_batch_destroy(ttm_batch* batch);

/* ------------------------------------------------------------ tracing */

/* Per-stage timing of a plan with CUDA events recorded on the stream of
 * each call (off by default). Stages: 0 prefilter + variance floor,
 * 1 image spectrum, 2 local sums -> w, 3 fused z pass, 4 y pass, 5 x pass
 * with the w epilogue, 6 peak map. ttm_plan_stage_times
 * synchronises, adds the elapsed milliseconds of every call since the last
 * reset into ms[0..n-1] (n <= ttm_num_stages()) and clears the record. */
ttm_status ttm_plan_enable_timing(ttm_plan* plan, int on);
ttm_status ttm_plan_stage_times(ttm_plan* plan, double* ms, int n);
int ttm_num_stages(void);
const char* ttm_stage_name(int i);

/* Number of kernels this library has launched in the process so far. */
uint64_t ttm_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* TTM_H */
