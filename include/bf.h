/*
 * libbf -- the trigonometric O(1) bilateral filter of Chaudhury, Sage and
 * Unser ("Fast O(1) bilateral filtering using trigonometric range kernels"),
 * as hand-written CUDA for GB300 (sm_103a).
 *
 * What every entry point computes (Section 1, eq. (BF) and
 * eq. (normalization), the unbiased form):
 *
 *     out(x) = sum_y w(y) phi(f(x-y) - f(x)) f(x-y) / sum_y w(y) phi(f(x-y) - f(x))
 *
 * with the raised-cosine range kernel of Section 2.3 scaled as in Algorithm 1
 * step 3 (rho = gamma sigma_r, gamma = pi/(2T)):
 *
 *     phi(s) = cos(s / (sigma_r sqrt(N)))^N
 *            = sum_{n=0..N} 2^-N C(N,n) exp(j (2n-N) s / (sigma_r sqrt(N)))
 *
 * evaluated through eq. (final-form): spatial averages of the auxiliary images
 * cos(w f), sin(w f), f cos(w f), f sin(w f), combined per pixel and divided.
 * The degree is N = max(1, ceil((gamma sigma_r)^-2)) (Algorithm 1 step 2,
 * Table 1).  The image is extended past its border by clamping coordinates to
 * the nearest edge pixel (the paper integrates over Omega and does not say).
 *
 * Conventions shared by all calls:
 *   - Every pointer named in/out/f/q/grad/workspace is a DEVICE pointer owned
 *     by the caller; the library never frees it.  Host pointers are named as
 *     such.  Images are row-major.
 *   - Calls that take a cudaStream_t are asynchronous on that stream; the
 *     returned status covers argument checks and launch errors only.
 *   - On any status other than BF_OK, bf_last_error() returns a message for
 *     the calling thread.  No call aborts the process.
 *   - Input values are expected in [0, T] (Section 2.1); they are not checked.
 */
#ifndef BF_H_
#define BF_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same definition as the CUDA runtime's; repeated so this header stands alone. */
typedef struct CUstream_st *cudaStream_t;

typedef enum {
    BF_OK = 0,
    BF_EINVAL = 1,         /* bad argument (NULL pointer, size, sigma, stride) */
    BF_EUNSUPPORTED = 2,   /* valid but outside what the kernels implement */
    BF_ECUDA = 3,          /* a CUDA runtime call or launch failed */
    BF_ENOMEM = 4,         /* host or device allocation failed */
    BF_ETIMEOUT = 5        /* a bounded device-side wait ran out */
} bf_status;

typedef enum {
    BF_SPATIAL_GAUSS_TRUNC = 0,  /* w1(i) ~ exp(-i^2 / 2 sigma_s^2), |i| <= R, unit sum */
    BF_SPATIAL_BOX_ITER = 1,     /* box_passes boxes of half-width r, convolved */
    BF_SPATIAL_GAUSS_RECURSIVE = 2
    /* The recursive O(1) Gaussian the paper's experiments use (Section 3): the
     * third-order causal + anticausal recursion of Young and van Vliet (1995)
     * with their published design q(sigma_s), b0..b3, applied along columns
     * and then rows; cost independent of sigma_s (0.5 <= sigma_s <= 256).
     * Borders (clamp-to-edge): the causal pass starts from its steady state
     * for the first sample, runs P = ceil(6 sigma_s) samples on into the
     * constant extension after the last one, and the anticausal pass starts
     * there from its steady state.  bf_plan_info reports P as the radius. */
} bf_spatial_kind;

typedef enum { BF_F32 = 0, BF_U8 = 1 } bf_dtype;

/*
 * How the plan picks the degree N when N_override is 0 (Algorithm 1 step 2:
 * "set N = (gamma sigma_r)^-2, or use a look-up table").
 *   BF_DEGREE_ESTIMATE: N = max(1, ceil((gamma sigma_r)^-2)), the smallest N
 *     that keeps every phase within [-pi/2, pi/2], so phi >= 0 and monotone
 *     on [0, T] (Section 2.4).
 *   BF_DEGREE_TABLE1: the empirical minimum degrees N_0 of Table 1 (T = 255;
 *     sigma_r in {200, 150, 100, 80, 60, 50, 40} -> N_0 = 1, 2, 3, 4, 5, 7, 9),
 *     applied at sigma' = 255 sigma_r / T (the approximation problem is the
 *     same after scaling s by 255 / T).  Between two tabulated values the plan
 *     takes the smaller of the N_0 listed for the next smaller tabulated sigma
 *     and the estimate; at sigma' >= 200, N = 1; below 40, where the table
 *     lists nothing, the estimate.  Such degrees let phases exceed pi/2: phi
 *     then takes values slightly below 0 (at most 3.6e-3 in magnitude, at
 *     sigma' = 60, N = 5), which the method reproduces exactly as it does any
 *     other trigonometric kernel; the caller accepts that P / Q is then no
 *     longer a convex combination.
 */
typedef enum { BF_DEGREE_ESTIMATE = 0, BF_DEGREE_TABLE1 = 1 } bf_degree_rule;

typedef struct {
    int N_override;      /* degree N; 0 = chosen by degree_rule */
    int radius_override; /* Gaussian: support half-width R (0 = ceil(3 sigma_s));
                            box: half-width r of one box (0 = the r whose
                            box_passes-fold variance is closest to sigma_s^2) */
    int box_passes;      /* box only; 0 = 3.  Only 3 is implemented. */
    int degree_rule;     /* bf_degree_rule; 0 = BF_DEGREE_ESTIMATE */
} bf_plan_opts;

/* Opaque, host-owned plan.  Creating one never touches a GPU. */
typedef struct bf_plan bf_plan;

/*
 * Algorithm 1 steps 1-3, on the host in double precision: the degree N, the
 * binomial coefficients 2^-N C(N,n) folded into one real weight per distinct
 * frequency |2n - N| / (sigma_r sqrt N), and the 1-D spatial taps.
 *   out      : receives the plan (host memory, free with bf_plan_destroy)
 *   sigma_s  : spatial standard deviation, > 0
 *   sigma_r  : range standard deviation, > 0
 *   T        : dynamic range bound of the image values, > 0 (255 for 8-bit)
 *   kind     : spatial kernel
 *   opts     : NULL for defaults
 * Errors: BF_EINVAL for non-positive or non-finite sigma/T, a NULL out, a
 *         negative option or an unknown degree_rule; BF_EUNSUPPORTED for
 *         N > 1024, a support radius above the kernels' limits, or
 *         box_passes other than 3.
 */
bf_status bf_plan_create(bf_plan **out, double sigma_s, double sigma_r, double T,
                         bf_spatial_kind kind, const bf_plan_opts *opts);

/*
 * A plan for a general trigonometric range kernel (Section 2.2, eq. (kernel)
 * in its real form):
 *     phi(s) = a[0] + a[1] cos(gamma s) + ... + a[N] cos(N gamma s),  N = n_coef - 1,
 * of which the raised cosine of bf_plan_create is one instance.  Everything
 * else -- spatial kernel, tile and streaming kernels, stacks, batches, the
 * backward pass for dL/df -- is shared with raised-cosine plans.
 *   sigma_s, kind, opts : as in bf_plan_create (opts->N_override and
 *                         opts->degree_rule must be 0)
 *   gamma               : base angular frequency in radians per gray level, > 0
 *   a                   : host array of n_coef real coefficients (copied)
 *   n_coef              : 1 <= n_coef <= 1025
 * Terms whose FP32 weight is 0 are dropped (they add exactly 0).  The caller
 * chooses a kernel that is positive on the range of differences the image
 * has (Section 2.1's conditions on a range kernel); otherwise the normaliser
 * Q can vanish.  bf_plan_info reports N as the highest n with a[n] != 0 in
 * FP32.  bf_backward and its variants reject grad_sigma_r for such a plan
 * (BF_EINVAL): it has no sigma_r.
 * Errors: BF_EINVAL for NULL pointers, gamma or sigma_s not finite and > 0,
 *         non-finite coefficients, all coefficients 0, or N_override or
 *         degree_rule set;
 *         BF_EUNSUPPORTED for n_coef > 1025 or a support beyond the kernels.
 */
bf_status bf_plan_create_cosine(bf_plan **out, double sigma_s, double gamma, const double *a,
                                int n_coef, bf_spatial_kind kind, const bf_plan_opts *opts);

void bf_plan_destroy(bf_plan *plan);

/*
 * Host-side facts about a plan (any output pointer may be NULL):
 *   N                : degree of the raised cosine
 *   n_freq           : number of terms the kernels evaluate: distinct nonzero
 *                      frequencies whose FP32 weight is not 0, plus one for
 *                      the constant term when N is even
 *   radius           : support half-width of the 2-D spatial kernel per axis
 *                      (R for the Gaussian, box_passes*r for the box; for the
 *                      recursive Gaussian the extension P past the last sample)
 *   achieved_sigma_s : standard deviation of the 1-D spatial kernel in use
 *                      (for the recursive Gaussian: of its impulse response)
 */
bf_status bf_plan_info(const bf_plan *plan, int *N, int *n_freq, int *radius,
                       double *achieved_sigma_s);

/*
 * The plan's term table in FP64 (host memory): for term k,
 *   a[k]     weight of cos(omega[k] (f(y) - f(x))) in phi, and
 *   omega[k] its angular frequency in radians per gray level.
 * Terms come in the order the kernels accumulate them (smallest weight first,
 * the constant term omega = 0 last).  sum_k a[k] cos(omega[k] s) = phi(s).
 * cap is the capacity of both arrays; *count receives the number of terms.
 */
bf_status bf_plan_terms(const bf_plan *plan, double *a, double *omega, int cap, int *count);

/* The 1-D spatial taps w1[0 .. 2*radius] in FP64 (host memory), unit sum. */
bf_status bf_plan_weights(const bf_plan *plan, double *w1, int cap, int *count);

/*
 * Fused forward filter (Algorithm 1 steps 3-5 in one kernel): the auxiliary
 * images are generated on chip from each tile of f, filtered on chip, and
 * combined in registers; HBM sees one read of f and one write of out.
 *   in               : device image, H x W x C interleaved (HWC), element type dt
 *   dt               : BF_F32 or BF_U8 (u8 is converted exactly to float)
 *   out              : device float image, H x W x C, row stride W*C
 *   H, W, C          : image size; H, W >= 1; 1 <= C <= 4; channels are
 *                      filtered independently with the same plan (Section 3)
 *   row_stride_elems : distance between rows of `in` in elements, >= W*C
 *   q_out            : NULL, or device float H x W x C receiving the
 *                      normaliser eq. (normalization) (unit-mass w), kept for
 *                      the backward pass
 *   stream           : CUDA stream
 * Kernels: the fused tile kernel serves the truncated Gaussian (R <= 24) and
 * the box with r <= 8.  For the box with 8 < r <= 64 the support does not fit
 * on chip and the filter runs as streaming sweeps (vertical, then horizontal)
 * through a scratch buffer of about (4 * terms + 2 * ceil(terms / 4) + 1) * H * W
 * floats (terms capped so that the vertical sweep's output stays within
 * 4 GiB); the recursive Gaussian streams the same way through about
 * 4 * terms * (H + P) * (W + P) floats.  The library allocates the scratch on
 * the current device the first time it is needed and keeps it for reuse
 * until bf_release_scratch(); the first such call on a device must therefore
 * not happen during stream capture.
 * Errors: BF_EINVAL (NULL pointers, sizes), BF_EUNSUPPORTED (C > 4),
 *         BF_ENOMEM (scratch allocation), BF_ECUDA (launch failure).
 */
bf_status bf_forward(const bf_plan *plan, const void *in, bf_dtype dt, float *out,
                     int H, int W, int C, long long row_stride_elems, float *q_out,
                     cudaStream_t stream);

/*
 * Space-variant extension (Section 4): the range kernel of `plan` with a
 * spatial kernel that changes from pixel to pixel -- pixel x averages over its
 * own (2 r(x) + 1) x (2 r(x) + 1) box of the clamp-extended image (equal
 * weights, which cancel in the ratio):
 *     out(x) = sum_{|y|_inf <= r(x)} phi(f(x-y) - f(x)) f(x-y)
 *              / sum_{|y|_inf <= r(x)} phi(f(x-y) - f(x)).
 * Computed through eq. (final-form) with per-term summed-area tables of the
 * four auxiliary images of the tile, O(1) per pixel and term whatever r(x).
 * Each tile of the output builds its tables over a halo of the largest r(x)
 * among its own pixels.  The tables hold 32-bit fixed-point values whose step
 * is set by that largest box and, for the f-weighted planes, by the value
 * range of the extended tile, so that every box sum comes out exact for the
 * fixed-point planes; the step's rounding error is of the order of the FP32
 * sine's.  Results therefore depend, to rounding, on the tile each pixel falls
 * in (its largest radius and its values), not only on r(x).
 * The plan's own spatial kernel is not used; its range kernel (raised cosine
 * or cosine polynomial) is.  Input values must be finite.
 *   in               : device image, H x W, single channel, type dt, rows
 *                      row_stride_elems (>= W) elements apart
 *   radius           : device int32 H x W, row-major (row stride W): the
 *                      half-widths r(x); values are clamped into [0, r_max]
 *   r_max            : 0 <= r_max <= 16, a bound on the half-widths (it
 *                      selects the kernel's largest halo and shared-memory
 *                      footprint; smaller is faster)
 *   out              : device float H x W, row stride W
 * Asynchronous on `stream`.  Errors: BF_EINVAL (NULL pointers, sizes,
 * r_max), BF_EUNSUPPORTED (image too large), BF_ECUDA (launch failure).
 */
bf_status bf_forward_space_variant(const bf_plan *plan, const void *in, bf_dtype dt,
                                   const int *radius, int r_max, float *out, int H, int W,
                                   long long row_stride_elems, cudaStream_t stream);

/*
 * The same with the hat of Section 4: pixel x weighs the clamp-extended image
 * at offset (a, b) by (r(x) + 1 - |a|) (r(x) + 1 - |b|), |a|, |b| <= r(x)
 * (the separable triangle of half-width r(x); its total weight cancels in the
 * ratio).  O(1) per pixel and term: per axis the hat is the second
 * difference, step r + 1, of a doubly integrated table, so each own pixel
 * reads nine entries of each of the four tables.  The tables hold 32-bit
 * fixed-point values whose every hat sum is exact.  r_max <= 8: with the hat's
 * weight (r + 1)^4 the fixed-point step of a 32-bit table above that would
 * let the rounding reach the 0.05 gray-level bar.  Arguments, layout and
 * errors as bf_forward_space_variant.
 */
bf_status bf_forward_space_variant_hat(const bf_plan *plan, const void *in, bf_dtype dt,
                                       const int *radius, int r_max, float *out, int H, int W,
                                       long long row_stride_elems, cudaStream_t stream);

/*
 * Both of the above for C interleaved channels (H x W x C, as bf_forward),
 * each filtered with the same radius map:
 *   spatial          : 0 the box (r_max <= 16), 1 the hat (r_max <= 8)
 *   in               : device image, type dt, rows row_stride_elems (>= W C)
 *                      elements apart, channel c of pixel (y, x) at
 *                      y row_stride_elems + x C + c
 *   out              : device float H x W x C, interleaved
 *   C                : 1 .. 4
 * bf_forward_space_variant(_hat) is this with C = 1.  Errors as
 * bf_forward_space_variant, plus BF_EINVAL for C or spatial out of range.
 */
bf_status bf_forward_space_variant_ex(const bf_plan *plan, const void *in, bf_dtype dt,
                                      const int *radius, int r_max, int spatial, float *out,
                                      int H, int W, int C, long long row_stride_elems,
                                      cudaStream_t stream);

/*
 * bf_forward for an image in HOST memory (not in the paper): in stream order,
 * copies host_in into the caller's device buffer dev_in, filters dev_in into
 * the caller's device buffer dev_out as bf_forward does, and copies dev_out
 * back into host_out.
 *   host_in  : host image laid out as bf_forward's `in` (H rows of
 *              row_stride_elems elements of type dt, the last row W*C long),
 *              or NULL when dev_in already holds the image (another filter of
 *              the same image: no copy)
 *   dev_in   : device buffer of at least ((H-1)*row_stride_elems + W*C)
 *              elements of type dt
 *   dev_out  : device float buffer of H*W*C elements
 *   host_out : host float buffer of H*W*C elements receiving the result, or
 *              NULL to leave it in dev_out only
 * The copies are cudaMemcpyAsync on `stream`: asynchronous (the call returns
 * before they finish) when the host buffers are page-locked
 * (cudaHostAlloc/cudaHostRegister), otherwise the runtime's pageable-copy
 * rules apply.  The host buffers must stay valid, and host_out unread, until
 * `stream` has reached the end of the call's work.  The library owns none of
 * the four buffers.  Errors: as bf_forward, plus BF_EINVAL for a NULL dev_in
 * or dev_out, BF_ECUDA for a failed copy.
 */
bf_status bf_forward_host(const bf_plan *plan, const void *host_in, bf_dtype dt, void *dev_in,
                          float *dev_out, float *host_out, int H, int W, int C,
                          long long row_stride_elems, cudaStream_t stream);

/*
 * bf_forward_host with the copy back on a second stream (not in the paper):
 * the copy in (when host_in is not NULL) and the filter run on `stream` as in
 * bf_forward_host; the copy of dev_out into host_out waits for this call's
 * filter on `copy_stream` only, so that `stream` goes on with the next
 * filter while the result travels.  host_out is complete once copy_stream
 * reaches the copy.  Later work must not write dev_out before the copy is
 * done: use another dev_out, or make `stream` wait for copy_stream.
 * copy_stream must differ from stream.  Errors as bf_forward_host.
 */
bf_status bf_forward_host_overlap(const bf_plan *plan, const void *host_in, bf_dtype dt,
                                  void *dev_in, float *dev_out, float *host_out, int H, int W,
                                  int C, long long row_stride_elems, cudaStream_t stream,
                                  cudaStream_t copy_stream);

/*
 * bf_forward over a stack of `count` single-channel images of one size, laid
 * out contiguously (image k at in + k*H*W elements, out + k*H*W floats),
 * all filtered with the same plan in one launch (channels are independent,
 * Section 3).  q_out, when not NULL, is a stack of the same shape.  Same
 * kernels, limits and errors as bf_forward; 1 <= count <= 65535.
 */
bf_status bf_forward_stack(const bf_plan *plan, const void *in, bf_dtype dt, float *out,
                           int H, int W, int count, float *q_out, cudaStream_t stream);

/*
 * Tile-shape autotuner for bf_forward (not in the paper).  Runs each tile
 * configuration the fused kernel has for this plan's spatial support `reps`
 * times on the given buffers (out is overwritten), and keeps the fastest for
 * later bf_forward calls with the same kind, radius, degree, H, W and C
 * (process-wide, thread-safe).  Synchronises `stream`.  *shape receives the
 * choice (-1 when the support runs on the streaming kernels, which have no
 * shape to choose), *ms its time per call; either may be NULL.  A
 * configuration is shape | split << 8.  Shape ids:
 *   0  32 x 64 tiles (every support)
 *   1  32 x 96 tiles, wider row segments (box r <= 4, Gaussian R <= 9)
 *   2  64 x 64 tiles, one 512-thread block per SM (box 3 <= r <= 8,
 *      Gaussian R >= 9)
 *   3  64 x 64 tiles, 32-pixel row segments, one 256-thread block per SM
 *      (box 7 <= r <= 8)
 * split (1, 2, 4, 8 or 16; 0 reads as 1): images
 * with fewer tiles than the GPU has SMs cut the terms into `split`
 * consecutive groups, one block per tile and group, so that the grid fills
 * the GPU; the groups of a tile run as one thread-block cluster whose blocks
 * each finish a slice of the tile, adding the groups' numerators and
 * normalisers (read from every block's shared memory) in group order.
 * Nothing is allocated.  The tuner and the default consider splits of the
 * 32-row shapes 0 and 1 (a cluster of the 64-row shapes' one-block-per-SM
 * blocks holds as many SMs); bf_forward_set_shape accepts any shape.
 * Without a tuned configuration bf_forward picks the split that brings the
 * blocks nearest two per SM.  Different configurations sum the terms in different orders, so
 * their results agree to FP32 rounding, not bit for bit; one configuration
 * gives the same bits run to run.
 */
bf_status bf_forward_tune(const bf_plan *plan, const void *in, bf_dtype dt, float *out, int H,
                          int W, int C, long long row_stride_elems, int reps,
                          cudaStream_t stream, int *shape, float *ms);

/*
 * Pins the tile configuration (shape | split << 8, as above) that later
 * bf_forward calls use for this plan's kind, radius and degree at size
 * H x W x C (C: the channels, or the images of a bf_forward_stack), as
 * bf_forward_tune would after timing.  Host only.  Errors:
 * BF_EINVAL for a shape the plan's support does not have (or a support
 * without tile shapes), a split that is not a power of two up to 8 or exceeds
 * the number of terms, or bad sizes.
 */
bf_status bf_forward_set_shape(const bf_plan *plan, int H, int W, int C, int shape);

/* Frees the scratch buffers bf_forward allocated (all devices).  Call only
 * when no work that uses them is in flight. */
void bf_release_scratch(void);

/*
 * The same filter, unfused: Algorithm 1 read literally (Section 2.2's
 * description of the O(1) algorithm), one term at a time -- the four
 * auxiliary images of the term are written to device memory, filtered by
 * separate kernels, and accumulated into numerator and denominator images in
 * device memory.  A baseline for the fused kernel; f32, one channel.
 *   workspace : device scratch of at least bf_forward_unfused_workspace(H, W)
 *               bytes, 256-byte aligned; contents on entry do not matter
 */
size_t bf_forward_unfused_workspace(int H, int W);
bf_status bf_forward_unfused(const bf_plan *plan, const float *in, float *out, int H,
                             int W, void *workspace, size_t workspace_bytes,
                             cudaStream_t stream);

/*
 * Adjoint of bf_forward for one f32 single-channel image (not in the paper:
 * the chain rule on eq. (BF), with the range-kernel derivative expanded in
 * the same trigonometric terms, and the spatial filter's adjoint -- the
 * filter itself in the interior, plus the clamped halo folded back onto the
 * edge pixels).  Given L = sum_x grad_out(x) out(x):
 *   f, out, q     : device H x W floats: the input and bf_forward's out, q_out
 *   grad_out      : device H x W floats, dL/d out
 *   grad_in       : device H x W floats, receives dL/df
 *   grad_sigma_r  : NULL, or a device double receiving dL/d sigma_r with N
 *                   held fixed (N is piecewise constant in sigma_r)
 *   workspace     : device scratch of bf_backward_workspace(plan, H, W) bytes
 *                   (needed only when grad_sigma_r is not NULL)
 * The planes are recomputed from f; nothing from the forward pass other than
 * out and q is stored.
 * Kernels: the fused adjoint tile kernel serves the truncated Gaussian
 * (R <= 24) and the box with r <= 8.  The box with 8 < r <= 64 runs the same
 * chain rule term by term through planes in device memory: about
 * 48 * H * W bytes of the library's scratch (the one bf_forward's
 * large-radius path uses, shared with it, allocated on first need and kept
 * until bf_release_scratch(); the first such call on a device must not
 * happen during stream capture).  That path is bandwidth-bound, not fused.
 * The recursive Gaussian (Section 3) takes the same path with its own line
 * filter and that filter's transpose (the recursions run in the same
 * directions from zero starts, the adjoints of the steady-state starts added
 * at the line's ends and the extension folded onto its last pixel), about
 * 48 * H * W + 24 * P * (H + W) bytes of that scratch, P = ceil(6 sigma_s).
 * Accuracy: dL/df within 1e-3 of the exact gradient (relative to its largest
 * element).  dL/dsigma_r carries the FP32 expansion's error in the kernel's
 * sigma_r-derivative weighted by grad_out / Q.  It stays within 1e-3 where Q
 * is not small, and within 1e-2 on images far smaller than the support
 * (tested down to 1 x 17 at r = 12).
 * Errors: BF_EINVAL (pointers, sizes, workspace, grad_sigma_r with a
 * cosine-polynomial plan), BF_EUNSUPPORTED (no adjoint for the support,
 * image too large), BF_ENOMEM (scratch), BF_ECUDA (launch failure).
 */
size_t bf_backward_workspace(const bf_plan *plan, int H, int W);
bf_status bf_backward(const bf_plan *plan, const float *f, const float *out,
                      const float *q, const float *grad_out, float *grad_in,
                      double *grad_sigma_r, int H, int W, void *workspace,
                      size_t workspace_bytes, cudaStream_t stream);

/*
 * bf_backward over a contiguous stack of `count` H x W images (layout as in
 * bf_forward_stack) in one launch (the box with r > 8: the stack's images
 * share each launch, in chunks of up to 2 GiB of scratch); grad_sigma_r
 * receives the sum over the stack of dL/dsigma_r (the images share sigma_r).  workspace needs
 * bf_backward_stack_workspace(plan, H, W, count) bytes, 8-byte aligned, when
 * grad_sigma_r is not NULL.
 */
size_t bf_backward_stack_workspace(const bf_plan *plan, int H, int W, int count);
bf_status bf_backward_stack(const bf_plan *plan, const float *f, const float *out,
                            const float *q, const float *grad_out, float *grad_in,
                            double *grad_sigma_r, int H, int W, int count, void *workspace,
                            size_t workspace_bytes, cudaStream_t stream);

/*
 * bf_backward for callers that cannot allocate device memory.  The paper has
 * no counterpart; this is a deployment variant of the adjoint above.  Some
 * callers cannot call cudaMalloc: code in a real-time loop, where an
 * allocation may synchronise the device and stall the frame; applications
 * whose memory pool is sized once at start-up and must not grow; plug-in
 * hosts (image editors, game engines) that own every device allocation and
 * hand the plug-in only its input and output buffers.  This entry point takes
 * the same arguments and gives the same results as bf_backward without the
 * workspace: the per-block partial sums of dL/dsigma_r go to a fixed array of
 * 16384 doubles (128 KiB) that is part of the library and stays resident on
 * every GPU that loads it until the process exits.
 *   Limit: with grad_sigma_r not NULL, ceil(W/64) * ceil(H/32) <= 16384
 *          (every image up to 4096 x 4096 fits); larger images return
 *          BF_EUNSUPPORTED with a message naming the limit.  With
 *          grad_sigma_r NULL no scratch is used and there is no limit.
 *   The first call on a device asks the runtime for the array's device
 *   address and caches it; make that first call before any stream capture.
 *   cudaDeviceReset on that device invalidates the cached address (the
 *   module is loaded again, possibly elsewhere): do not call this entry
 *   point on a device after resetting it in the same process.
 *   All calls share the array.  Each call writes every partial it reads
 *   before reading it, so nothing has to be cleared between calls, but calls
 *   whose work overlaps on the GPU (other streams, other host threads) race
 *   on the array: serialise them.
 *   Supports: the fused adjoint's (Gaussian R <= 24, box r <= 8); the box
 *   with r > 8 and the recursive Gaussian need device scratch and return
 *   BF_EUNSUPPORTED here.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 */
bf_status bf_backward_noalloc(const bf_plan *plan, const float *f, const float *out,
                              const float *q, const float *grad_out, float *grad_in,
                              double *grad_sigma_r, int H, int W, cudaStream_t stream);

/*
 * Batched forward: many f32 single-channel images of uneven sizes, each with
 * its own plan (own sigma_s, sigma_r and hence N), replayed from one CUDA
 * graph.  Images whose box half-width fits a tile (r <= 8) share ONE
 * persistent launch that pulls work items (a tile, or a tile's group of
 * terms) from a device work queue, largest cost first; each radius bucket
 * r = 1 .. 8 has its own configuration (tile shape and term split, see
 * bf_batch_set_config), and the term groups of split images are summed in
 * group order by one more kernel.  Images with 8 < r <= 64, and images whose
 * plan is the recursive Gaussian, run the streaming sweeps of bf_forward in
 * the same graph, in up to four concurrent chains
 * (images spread over the chains largest cost first), concurrently with the
 * persistent launch.  Each image's result is bit-identical to bf_forward's
 * in the same configuration (bf_forward_set_shape with the bucket's shape
 * and split).
 *
 * bf_batch_create  : plans[count], H[count], W[count] are host arrays; the
 *                    batch copies what it needs (the plans may be destroyed
 *                    afterwards).  Every plan must be the 3-pass box with
 *                    1 <= r <= 64 or the recursive Gaussian
 *                    (BF_EUNSUPPORTED otherwise).  Allocates the batch's
 *                    device tables, queue and, if some image streams, one
 *                    scratch per chain of streaming images (the largest
 *                    bf_forward scratch among the chain's images); all freed
 *                    by bf_batch_destroy.
 * bf_batch_bind    : in[count], out[count] are host arrays of device
 *                    pointers (f32, row stride W); copied to the device on
 *                    `stream`, which is synchronised; the graph is captured
 *                    again (on a private stream of the batch).  Call again
 *                    whenever the buffers change.
 * bf_batch_forward : replays the graph on `stream` (allocates nothing).
 * bf_batch_check   : waits for `stream` and reports the device error flag
 *                    (non-zero if a tile-queue bound was hit).
 */
typedef struct bf_batch bf_batch;
bf_status bf_batch_create(bf_batch **out, const bf_plan *const *plans, const int *H,
                          const int *W, int count);
bf_status bf_batch_bind(bf_batch *batch, const float *const *in, float *const *out,
                        cudaStream_t stream);
bf_status bf_batch_forward(bf_batch *batch, cudaStream_t stream);
bf_status bf_batch_check(bf_batch *batch, cudaStream_t stream, int *device_error);
void bf_batch_destroy(bf_batch *batch);

/*
 * Configuration of radius bucket r (1 <= r <= 8) of a batch (not in the
 * paper): the tile shape of its images (ids as bf_forward_tune's, all with
 * 256 threads per tile: 0 = 32 x 64 tiles, 8 pixels per thread; 1 = 32 x 96,
 * 12 pixels per thread, r <= 4; 3 = 64 x 64, 16 pixels per thread,
 * r = 7, 8) and the number of groups its terms are cut into (1, 2 or 4, each
 * group of a tile a separate work item; split images keep their groups'
 * numerators and normalisers in a batch-owned buffer of 2 * split * H * W
 * floats).  bf_batch_config reads it (host only); bf_batch_set_config sets
 * it, synchronises `stream`, re-uploads the batch's tables and captures its
 * graph again.  Defaults: shape 0, split 1.  Errors: BF_EINVAL for r outside
 * 1 .. 8, a shape the bucket does not have, a split other than 1, 2, 4.
 */
bf_status bf_batch_config(const bf_batch *batch, int r, int *shape, int *split);
bf_status bf_batch_set_config(bf_batch *batch, int r, int shape, int split,
                              cudaStream_t stream);

/*
 * Autotuner for a bound batch (not in the paper): for each radius bucket of
 * tiled images in turn (largest share of the tile work first), every tile
 * shape the bucket has and every term split (1, 2, 4), the other buckets as
 * they stand, each timed as the fastest of 2 reps + 1 launches of the tiled
 * images alone; then the persistent grid (1x or 2x the resident blocks) and
 * the queue order (largest cost first or image order), each timed as the
 * fastest of `reps` replays of the whole batch, streaming images (r > 8)
 * included.  A candidate replaces the configuration in hand only when more
 * than 1 % faster.  The result is kept in the batch's graph (bf_batch_config
 * reads the buckets' choices) and the grid, order and whole-batch time
 * reported (any output may be NULL).  Synchronises `stream`.
 */
bf_status bf_batch_tune(bf_batch *batch, cudaStream_t stream, int reps, int *grid,
                        int *order, float *ms);

/*
 * Measured FP32 FMA-pipe throughput of the current device (not in the paper;
 * a measuring aid, not part of the filter).  The filter's kernels are bound by
 * plain FP32 arithmetic, so their roofline denominator is the rate of FP32
 * lane operations.  This call launches a kernel of independent FMA chains on
 * every SM (2048 resident threads each; paired != 0: FFMA2, two lane
 * operations per instruction), times five launches after two warm-up launches
 * with CUDA events on `stream`, synchronises `stream` and stores lane
 * operations per second (an FFMA counts as one) in the HOST double
 * *lane_ops_per_s.  About 10 ms of GPU time.  BF_EINVAL for a NULL output,
 * BF_ECUDA for a failed launch or event.
 */
bf_status bf_fp32_pipe_rate(int paired, double *lane_ops_per_s, cudaStream_t stream);

/* Message for the last non-OK status returned on the calling thread. */
const char *bf_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int bf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BF_H_ */
