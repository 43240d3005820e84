/*
 * fht.h -- C ABI of the GB300 (sm_103a) library for the Brady dyadic fast Hough
 * transform and the modifications of Aliev, Ershov and Nikolaev, "On the use
 * of FHT, its modification for practical applications and the structure of
 * Hough image" (arXiv:1811.06378).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images are row-major, h rows by w columns, element (y, x) at
 * base[y * pitch + x]; every pitch is counted in ELEMENTS of the buffer's own
 * type and must be >= the row length. Every data pointer is a DEVICE pointer
 * (CUDA global memory) unless a comment says "host". `stream` is a
 * cudaStream_t passed as void* (NULL = the legacy default stream). All calls
 * that take a stream are asynchronous on it; argument checks happen on the
 * host before anything is enqueued, and a call that returns an error has
 * enqueued nothing.
 *
 * Ownership: the caller allocates and frees every device buffer, including
 * the workspace (scratch for intermediate butterfly levels) whose size the
 * *_workspace_size queries return. The library allocates no device memory at
 * call time (fht_forward_static's fixed array is part of the loaded library).
 * A workspace may be reused by calls that are ordered on one stream; calls
 * running concurrently need separate workspaces. Full-layout calls may run
 * their quadrants on streams of the library's own, forked from and joined
 * back into the caller's stream (fht_full_quadrants).
 *
 * Errors: status codes only; nothing is thrown across the ABI.
 *   FHT_EINVAL        bad sizes, pitches, dtypes, slope ranges, null pointers,
 *                     or a workspace smaller than required
 *   FHT_ECUDA         a CUDA launch or copy failed (see fht_last_cuda_error)
 *   FHT_EUNSUPPORTED  a valid request this build does not implement
 *   FHT_ETIMEOUT      a device-side bounded wait gave up (batched kernel)
 *   FHT_EBOUNDS       the debug build refused an access outside a pass's
 *                     buffers (fht_device_status)
 *
 * Geometry (Section 3.1): for the mostly-vertical quadrants Q0/Q1 the image is
 * zero-padded virtually to n = next_pow2(h) rows and W = w + n columns taken
 * cyclically; the quadrant has n slope rows t = 0..n-1 (t = n-1 is 45 deg) and
 * W columns. The mostly-horizontal quadrants Q2/Q3 are the same on the
 * transposed image: n = next_pow2(w), W = h + n. Padding is never stored.
 *
 * The transform (Brady's recursion, cited by the paper in Section 2 and drawn
 * in Section 4, Figure 6): H_sigma[t][x] = sum_{y<n} P[y][(x + sigma*off_n(t,y)) mod W],
 * off_n(t,y) = sum_{j=1..K} bit_{K-j}(y) * ceil(floor(t/2^(j-1))/2), n = 2^K.
 * Q0 = sigma +1 on the image, Q1 = sigma -1 on the image, Q2 = sigma -1 on the
 * transposed image, Q3 = sigma +1 on the transposed image.
 *
 * Supported (input -> accumulator) types: u8->i32, i32->i32, u8->f32, f32->f32.
 * Integer accumulation wraps modulo 2^32 (exact while the true sums fit);
 * FP32 accumulation adds exactly the two operands the recursion names, in
 * round-to-nearest, so results are reproducible bit for bit.
 */
#ifndef FHT_H
#define FHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FHT_OK = 0,
    FHT_EINVAL = 1,
    FHT_ENOMEM = 2,
    FHT_ECUDA = 3,
    FHT_EUNSUPPORTED = 4,
    FHT_ETIMEOUT = 5,
    FHT_EBOUNDS = 6
} fht_status;

typedef enum { FHT_U8 = 0, FHT_I32 = 1, FHT_F32 = 2 } fht_dtype;

/* Angle quadrants of Section 3.1: Q0 [-45,0] deg (mostly vertical, positive
 * shift), Q1 [0,45], Q2 [45,90] (mostly horizontal), Q3 [90,135]. */
typedef enum { FHT_Q0 = 0, FHT_Q1 = 1, FHT_Q2 = 2, FHT_Q3 = 3 } fht_quadrant;

/* Layout of a Hough image: one quadrant (n x W), or the full image of
 * Section 3.3 (all four quadrants on a power-of-two-padded image). */
typedef enum { FHT_LAYOUT_QUADRANT = 0, FHT_LAYOUT_FULL = 1 } fht_layout;

/* Human-readable name of a status code (static string, never NULL). */
const char *fht_status_string(fht_status s);

/* The last CUDA error code seen by this library on the calling thread
 * (cudaError_t as int; 0 if none). */
int fht_last_cuda_error(void);

/* ------------------------------------------------------------------ geometry
 * Host-only, synchronous, no device access. */

/* Shape of quadrant q of an h x w image (Section 3.1): *rows = n, *cols = W. */
fht_status fht_query_shape(int h, int w, fht_quadrant q, int *rows, int *cols);

/* Shape of the full Hough image (Section 3.3): the image is padded to
 * h_p x w_p (next powers of two); *rows = 2*(h_p + w_p) - 3, *cols = h_p + w_p. */
fht_status fht_full_shape(int h, int w, int *rows, int *cols);

/* Which quadrant and slope a full-image row holds (Section 3.3, end): rows
 * [0, h_p) are Q0 flipped (t = h_p-1-row), then Q1 t = 1..h_p-1, then Q2
 * flipped t = w_p-2..0, then Q3 t = 1..w_p-1 (each seam's shared row kept once). */
fht_status fht_full_row_to_quadrant(int h, int w, int row, int *q, int *t);

/* Slope ranges for line angles in [phi_lo_deg, phi_hi_deg] (Section 4).
 * Quadrant spans Q0 [-45,0], Q1 [0,45], Q2 [45,90], Q3 [90,135]; inside a
 * quadrant with n slopes, slope t lies atan(t/(n-1)) away from the quadrant's
 * t = 0 edge (0 deg for Q0/Q1, 90 deg for Q2/Q3) and is kept iff that angle is
 * in the range. A seam row shared by two quadrants is kept in the first of
 * Q0, Q1, Q2, Q3. t_lo[q] = t_hi[q] = -1 marks an unused quadrant.
 * t_lo and t_hi are HOST arrays of 4 ints. */
fht_status fht_angle_to_slopes(double phi_lo_deg, double phi_hi_deg, int h, int w,
                               int *t_lo, int *t_hi);

/* Bytes of device workspace needed by fht_forward, fht_forward_range,
 * fht_full_quadrants and fht_adjoint on an h x w image with this layout,
 * quadrant (ignored for FHT_LAYOUT_FULL) and type pair. May be 0.
 * For FHT_LAYOUT_FULL it is one slice per quadrant, which lets the four
 * quadrants run concurrently (the library's default schedule;
 * FHT_CONCURRENT=0 in the environment when the library loads turns it off);
 * any workspace down to the largest single quadrant's is accepted and runs
 * the quadrants one after another. */
fht_status fht_workspace_size(int h, int w, fht_layout layout, fht_quadrant q,
                              fht_dtype in_t, fht_dtype acc_t, size_t *bytes);

/* ------------------------------------------------------------------ forward */

/* One quadrant of the Hough image (Sections 3.1-3.2).
 * img  h x w image of type in_t, pitch in_pitch.
 * out  n x W Hough image of type acc_t, pitch out_pitch >= W; row t = slope t,
 *      column x = x0 of Section 3.1 (cyclic over the padded width). */
fht_status fht_forward(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                       fht_quadrant q, void *out, fht_dtype acc_t, int64_t out_pitch,
                       void *workspace, size_t workspace_bytes, void *stream);

/* The angle-range variant (Section 4): only slopes t_lo..t_hi of quadrant q,
 * computed by pruning the slope index space at every butterfly level (the
 * levels compute only the slopes those outputs depend on). out has
 * t_hi - t_lo + 1 rows of W columns; row k holds slope t_lo + k, bit-identical
 * to row t_lo + k of fht_forward. 0 <= t_lo <= t_hi < n. */
fht_status fht_forward_range(const void *img, fht_dtype in_t, int h, int w,
                             int64_t in_pitch, fht_quadrant q, int t_lo, int t_hi,
                             void *out, fht_dtype acc_t, int64_t out_pitch,
                             void *workspace, size_t workspace_bytes, void *stream);

/* The full Hough image (Section 3.3): the image is padded to h_p x w_p, the
 * four quadrants are computed with width h_p + w_p, and their rows are written
 * straight into the concatenated layout (Q0 flipped, Q1, Q2 flipped, Q3; one
 * copy of each shared seam row). out is fht_full_shape rows x cols.
 * apply_fhtshift != 0 additionally rotates every row as fhtshift does
 * (Section 5), fused into the same stores.
 * With a workspace of fht_workspace_size bytes and the concurrent schedule on,
 * the quadrants run on the caller's stream and three streams of the library,
 * forked from and joined back into `stream` with events (stream capture turns
 * them into graph branches); work enqueued on `stream` afterwards still sees
 * the whole result. The library's streams are shared by every call on a
 * device: do not run such a call on one host thread while another thread is
 * capturing one. */
fht_status fht_full_quadrants(const void *img, fht_dtype in_t, int h, int w,
                              int64_t in_pitch, void *out, fht_dtype acc_t,
                              int64_t out_pitch, int apply_fhtshift, void *workspace,
                              size_t workspace_bytes, void *stream);

/* fhtshift (Section 5): rotate every row of a Hough image so that its
 * meaningful pixels form one run centred in the row, the black zone split to
 * both edges. Row t of a quadrant with black-zone width b = W - w_in - t
 * (w_in = w for Q0/Q1, h for Q2/Q3; w_p or h_p in the full layout) moves
 * right by floor(b/2) + t for the positive-sign quadrants Q0/Q3 and by
 * floor(b/2) for Q1/Q2; inverse != 0 undoes it. Out of place only
 * (in and out must not overlap). h, w are the IMAGE's sizes; the Hough image's
 * shape follows from them and the layout (q is ignored for the full layout).
 * dtype FHT_I32 or FHT_F32. */
fht_status fhtshift(const void *in, void *out, fht_dtype dtype, int h, int w,
                    fht_layout layout, fht_quadrant q, int inverse, int64_t in_pitch,
                    int64_t out_pitch, void *stream);

/* fht_forward for callers that cannot allocate device memory. The paper has
 * no counterpart; this is a property of the library, not of the method.
 * Some callers cannot call cudaMalloc or anything that allocates: code
 * confined to a memory pool or budget it does not own (a framework's caching
 * allocator, a real-time path with a fixed memory budget), plugin hosts that
 * forbid allocation after start-up. This entry point computes exactly what fht_forward computes (same
 * arguments, minus the workspace) but keeps the intermediate butterfly levels
 * in a fixed 64 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits. It allocates nothing.
 *
 * Limit: requests for which fht_workspace_size(h, w, FHT_LAYOUT_QUADRANT, q,
 * in_t, acc_t) exceeds 64 MiB return FHT_ENOMEM and enqueue nothing (a uint8
 * image up to 4096 x 4096 into int32 fits, with the default tuning).
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. A context that is torn down and created again
 * (cudaDeviceReset) holds the array at a new address: the first call in the
 * new context looks it up again, so it too should come before any capture.
 * Sharing: all calls on a device share the one array, which keeps the last
 * call's contents (nothing in it needs to start at zero). Calls whose kernels
 * overlap on the GPU race on it: issue them in order on one stream. */
fht_status fht_forward_static(const void *img, fht_dtype in_t, int h, int w,
                              int64_t in_pitch, fht_quadrant q, void *out,
                              fht_dtype acc_t, int64_t out_pitch, void *stream);

/* ------------------------------------------------------------------ adjoint */

/* Adjoint (transpose) of fht_forward (layout QUADRANT, quadrant q) or of
 * fht_full_quadrants without fhtshift (layout FULL): back-projects a Hough
 * image gradient onto the h x w image. Not in the paper: the transform is
 * linear and this is its exact transpose, run as the butterfly levels in
 * reverse (each merge becomes a split). grad_hough has the forward output's
 * shape, type dtype (FHT_F32 or FHT_I32), pitch in_pitch; grad_img is h x w
 * of the same type, pitch out_pitch, fully overwritten. For the full layout the
 * four quadrant contributions are summed in the order Q0, Q1, Q2, Q3 (also
 * under the concurrent schedule of fht_full_quadrants, where the passes before
 * each quadrant's final one overlap and the final passes stay in order). */
fht_status fht_adjoint(const void *grad_hough, fht_dtype dtype, int h, int w,
                       fht_layout layout, fht_quadrant q, int64_t in_pitch,
                       void *grad_img, int64_t out_pitch, void *workspace,
                       size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------ other operations
 * Hough transforms generalise to any associative-commutative operation along
 * the lines (the paper's introduction). The same recursion with the maximum
 * or the minimum in place of the sum: each level takes op(top, shifted
 * bottom). The padding is the zero-filled extension of Section 3.1 for every
 * operation, so a pattern that leaves the image takes zeros into its maximum
 * or minimum. */
typedef enum { FHT_OP_SUM = 0, FHT_OP_MAX = 1, FHT_OP_MIN = 2 } fht_op;

/* Slope rows t_lo..t_hi of quadrant q with operation op, layout and
 * arguments as fht_forward_range (op FHT_OP_SUM is fht_forward_range).
 * FHT_OP_MAX / FHT_OP_MIN take uint8 -> int32 (uint16 intermediate levels) or
 * float32 -> float32, else FHT_EUNSUPPORTED; the workspace
 * fht_workspace_size gives for the same types is enough. Exact for integers;
 * float32 maxima and minima are exact too (each result is one of the
 * inputs or zero). */
fht_status fht_forward_op(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                          fht_quadrant q, fht_op op, int t_lo, int t_hi, void *out,
                          fht_dtype acc_t, int64_t out_pitch, void *workspace,
                          size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------ back to lines
 * Host only: the image segment that Hough point (row, col) sums (Section 3.2).
 * The point's pattern (the dyadic digital line of its slope, from its column)
 * is taken with columns modulo the extended width W (a pattern that leaves
 * the extended image on the right re-enters the image on the left: the
 * paper's case b) and cut to the h x w image (case a). Its in-image pixels are
 * one run along the pattern: *count receives their number (0 when the
 * pattern lies wholly in the padding: case c, and the ends are -1), (r0, c0)
 * and (r1, c1) the image row and column of its first and last pixel in the
 * pattern's order (down the rows for Q0/Q1, along the columns for Q2/Q3).
 * layout FHT_LAYOUT_QUADRANT: row = slope t of quadrant q, col in [0, W).
 * layout FHT_LAYOUT_FULL: row = a row of the full image (q ignored; the
 * quadrants of the power-of-two-padded image, Section 3.3), col in
 * [0, h_p + w_p). shifted != 0: the Hough image had fhtshift applied
 * (Section 5); its rotation is undone first. */
fht_status fht_segment(int h, int w, fht_layout layout, fht_quadrant q, int row, int col,
                       int shifted, int *count, int *r0, int *c0, int *r1, int *c1);

/* Per-row maxima of a Hough image (rows x cols, int32 or float32, pitch in
 * elements): max_out[r] (rows values of dtype) and arg_out[r] (int32) the
 * largest value of row r and the first column holding it; the strongest line
 * of each slope. One read of the image; NaN entries give unspecified results.
 * Not in the paper. */
fht_status fht_row_argmax(const void *hough, fht_dtype dtype, int rows, int cols, int64_t pitch,
                          void *max_out, int *arg_out, void *stream);

/* ------------------------------------------------------------ sheared (Section 4)
 * The paper's way to a chosen range of line angles: shear the image
 * horizontally by spl (the shift per line) inside the first butterfly
 * iteration, then run one quadrant. Row y of the image (of the transposed
 * image for Q2/Q3) is taken as rotated right by s(y) = floor(y*spl + 1/2)
 * columns modulo W (the paper fixes no rounding; it is evaluated exactly with
 * spl in fixed point, P = floor(spl * 2^32 + 1/2), s(y) = (y*P + 2^31) >> 32),
 * zero outside the image, so that
 *   Hs[t][x] = sum_{y<n} P[y][(x + sigma*off_n(t,y) - s(y)) mod W].
 * A line with dx/dy = k then lies on slope k + spl: the quadrant's slopes
 * t/(n-1) in [0, 1] cover k in [-spl, 1 - spl] (Q0; columns per row of the
 * transposed image for Q2/Q3). The shear moves the black zone, so every
 * intermediate level is all W columns wide (cyclic); no fhtshift. */

/* Workspace bytes of fht_forward_sheared for this size, quadrant and types. */
fht_status fht_workspace_size_sheared(int h, int w, fht_quadrant q, fht_dtype in_t,
                                      fht_dtype acc_t, size_t *bytes);

/* Slope rows t_lo..t_hi of the sheared quadrant q into out ((t_hi - t_lo + 1)
 * x W, pitch out_pitch >= W; row t at out row t - t_lo); -1 <= spl <= 1
 * (FHT_EINVAL otherwise, NaN included); types as fht_forward. Only the slopes
 * those rows depend on are computed (the range pruning of fht_forward_range).
 * spl = 0 gives exactly fht_forward_range. */
fht_status fht_forward_sheared(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                               fht_quadrant q, double spl, int t_lo, int t_hi, void *out,
                               fht_dtype acc_t, int64_t out_pitch, void *workspace,
                               size_t workspace_bytes, void *stream);

/* One sheared quadrant for the line angles [phi_lo, phi_hi] (degrees, the
 * quadrant spans of fht_angle_to_slopes), host only. A mostly vertical range
 * (inside [-45, 45]) gives Q0 and spl = tan(phi_hi): row t holds the angle
 * atan(spl - t/(n-1)), phi_hi at t = 0. A mostly horizontal range (inside
 * [45, 135]) gives Q3 and spl = -tan(phi_lo - 90): row t holds
 * 90 + atan(t/(n-1) - spl), phi_lo at t = 0. t_lo = 0 and t_hi =
 * floor((n-1)*(tan(b) - tan(a))), a, b the range's ends measured from the
 * axis. FHT_EINVAL if the range crosses 45 or 135 degrees or its ends differ
 * by more than 1 in tangent. */
fht_status fht_shear_range(double phi_lo, double phi_hi, int h, int w, fht_quadrant *q,
                           double *spl, int *t_lo, int *t_hi);

/* ------------------------------------------------------------ scaled (Section 4)
 * The paper's other operation for a chosen range of angles: the image scaled
 * along its rows by alpha > 0 (for Q2/Q3 the rows of the transposed image,
 * i.e. the original scaled along OY) inside the first butterfly iteration; a
 * line with dx/dy = k becomes one with dx/dy = alpha*k. The paper fixes no
 * discrete resampling; this library takes nearest neighbour on the integer
 * grid, in fixed point so that it is exact and reproducible: with
 * D = ceil(2^32 / alpha) (the quotient in double), column c of the scaled row
 * is image column (c * D) >> 32 (floor(c / k) for an integer factor k: every
 * column repeated k times; k*c for alpha = 1/k), for the
 * w_alpha = ceil(w * 2^32 / D) columns whose source lies in the row. The
 * shear of fht_forward_sheared then applies to the scaled rows (scale first,
 * then shear), on the cyclic width W = w_alpha + n:
 *   Hs[t][x] = sum_{y<n} S[y][(x + sigma*off_n(t,y) - s(y)) mod W],
 * S the scaled image zero-padded to W columns. A line with dx/dy = k lies on
 * slope alpha*k + spl. Every intermediate level is all W columns wide. The
 * library writes S once into the workspace (one gather kernel) and runs the
 * sheared transform on it: the same sums as scaling inside the first
 * iteration, with the first pass reading whole vectors. */

/* Scaled width w_alpha of a row of w pixels (HOST). FHT_EINVAL unless
 * 1/256 <= alpha <= 256 and 1 <= w_alpha <= 32768. */
fht_status fht_scaled_width(int w, double alpha, int *w_alpha);

/* Shape (rows n, cols W = w_alpha + n) of the scaled quadrant q of an h x w
 * image; w_alpha scales w for Q0/Q1 and h for Q2/Q3. */
fht_status fht_scaled_shape(int h, int w, fht_quadrant q, double alpha, int *rows, int *cols);

/* Workspace bytes of fht_forward_scaled for this size, quadrant, factor and
 * types: the intermediate levels and, after them, the scaled copy of the
 * image the first pass reads (h x w_alpha for Q0/Q1, w_alpha x w for Q2/Q3,
 * rows padded to 16 bytes). */
fht_status fht_workspace_size_scaled(int h, int w, fht_quadrant q, double alpha,
                                     fht_dtype in_t, fht_dtype acc_t, size_t *bytes);

/* Slope rows t_lo..t_hi of quadrant q of the image scaled by alpha and then
 * sheared by spl (-1 <= spl <= 1; spl = 0: no shear) into out
 * ((t_hi - t_lo + 1) x W, pitch out_pitch >= W, row t at out row t - t_lo);
 * W from fht_scaled_shape; types as fht_forward. Only the slopes those rows
 * depend on are computed. alpha = 1 gives exactly fht_forward_sheared.
 * FHT_EINVAL for factors or sizes fht_scaled_shape rejects. */
fht_status fht_forward_scaled(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                              fht_quadrant q, double alpha, double spl, int t_lo, int t_hi,
                              void *out, fht_dtype acc_t, int64_t out_pitch, void *workspace,
                              size_t workspace_bytes, void *stream);

/* One scaled and sheared quadrant for the line angles [phi_lo, phi_hi]
 * (degrees), host only: the two operations map the range onto as many slope
 * rows as |spl| <= 1 allows, resolving its angles alpha times finer than the
 * plain quadrant. A mostly vertical range (midpoint in [-45, 45], ends inside
 * (-90, 90)) gives Q0 with alpha = min(1/(tan b - tan a), 1/|tan b|, 16),
 * spl = alpha*tan b, and row t holding atan((spl - t/(n-1))/alpha) (phi_hi
 * at t = 0), a = phi_lo, b = phi_hi. A mostly horizontal one (midpoint in
 * (45, 135], ends inside (0, 180)) gives Q3 with a, b measured from 90
 * degrees, alpha = min(1/(tan b - tan a), 1/|tan a|, 16), spl = -alpha*tan a,
 * and row t holding 90 + atan((t/(n-1) - spl)/alpha) (phi_lo at t = 0).
 * t_lo = 0, t_hi = floor((n-1) * alpha * (tan b - tan a)). FHT_EINVAL
 * otherwise. */
fht_status fht_scale_range(double phi_lo, double phi_hi, int h, int w, fht_quadrant *q,
                           double *alpha, double *spl, int *t_lo, int *t_hi);

/* ------------------------------------------------------------ one image over P GPUs
 * Not in the paper: how one quadrant splits over P = 2, 4 or 8 ranks by rows
 * (by columns of the original image for Q2/Q3). With n = 2^K slope rows and
 * W columns (fht_query_shape of the whole image), rank p holds the image rows
 * [p*n/P, (p+1)*n/P) (those below the image are absent: an empty or short
 * strip), and:
 *   1. fht_forward_padded: its strip's K - log2(P) levels, i.e. the strip's
 *      quadrant padded to n_s = n/P rows on the whole image's cyclic width W:
 *      n_s x W, row tau = the strip's slope tau;
 *   2. one all-to-all: rank b receives rows [b*n_s/P, (b+1)*n_s/P) of every
 *      strip's result (n_s/P x W per pair);
 *   3. fht_merge_strips: the last log2(P) levels on those rows, giving the
 *      quadrant's slope rows [b*n/P, (b+1)*n/P), bit for bit what one GPU
 *      computes (the same additions in the same order).
 * The Python package's `sharded` module runs the three steps over
 * torch.distributed. */

/* Workspace bytes of fht_forward_padded. */
fht_status fht_workspace_size_padded(int h, int w, fht_quadrant q, int n, int W,
                                     fht_dtype in_t, fht_dtype acc_t, size_t *bytes);

/* Quadrant q of the h x w image zero-padded to n rows (of the transposed image
 * for Q2/Q3; n a power of two, n >= those rows) and taken on the cyclic width
 * W >= w_c + n (w_c = w for Q0/Q1, h for Q2/Q3): n x W into out (pitch
 * out_pitch >= W); types as fht_forward. With n = next_pow2(rows) and
 * W = w_c + n this is fht_forward. The strip's row count may be 0 (an empty
 * strip: out is zeroed). */
fht_status fht_forward_padded(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                              fht_quadrant q, int n, int W, void *out, fht_dtype acc_t,
                              int64_t out_pitch, void *workspace, size_t workspace_bytes,
                              void *stream);

/* The last log2(strips) levels (strips = P = 1, 2, 4 or 8) for the slopes
 * tau = tau0 .. tau0 + rows - 1: parts holds, for each strip p, its level
 * rows tau (rows x W, pitch in_pitch) at parts + p * part_stride (elements);
 * out receives rows tau*P + c (c < P) at row (tau - tau0)*P + c (rows*P x W,
 * pitch out_pitch). dtype FHT_I32 or FHT_F32 (the accumulator); the sign is
 * quadrant q's. */
fht_status fht_merge_strips(const void *parts, fht_dtype dtype, int strips, int rows, int W,
                            int64_t part_stride, int64_t in_pitch, int tau0, fht_quadrant q,
                            void *out, int64_t out_pitch, void *stream);

/* ------------------------------------------------------------ uniform batches
 * `batch` transforms of the same size and layout in one launch per pass (the
 * launch's third grid dimension is the image), so that many small images fill
 * the GPU. Not in the paper; the differentiable path uses it for (B, h, w)
 * tensors. FP32 only (images, Hough images and gradients are float32).
 * Image b lies b * *_batch_stride ELEMENTS past image 0 (strides at least one
 * image apart: h * in_pitch for images, rows * out_pitch for Hough images);
 * 1 <= batch <= 65535. Layout FHT_LAYOUT_QUADRANT transforms quadrant q;
 * FHT_LAYOUT_FULL the four quadrants as fht_full_quadrants (without
 * fhtshift). Results equal the single-image calls bit for bit. */

/* Workspace bytes of a uniform batch: for each image, the bytes
 * fht_workspace_size(h, w, layout, q, FHT_F32, FHT_F32) returns, rounded up
 * to a multiple of 256. */
fht_status fht_workspace_size_many(int batch, int h, int w, fht_layout layout, fht_quadrant q,
                                   size_t *bytes);

/* Forward transform of a uniform batch: img -> out, as fht_forward (layout
 * QUADRANT) or fht_full_quadrants (layout FULL) for every image. */
fht_status fht_forward_many(const void *img, int batch, int64_t img_batch_stride, int h, int w,
                            int64_t in_pitch, fht_layout layout, fht_quadrant q, void *out,
                            int64_t out_batch_stride, int64_t out_pitch, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Adjoint of a uniform batch: grad_hough -> grad_img, as fht_adjoint for
 * every image (grad_img fully overwritten). */
fht_status fht_adjoint_many(const void *grad_hough, int batch, int64_t grad_batch_stride, int h,
                            int w, fht_layout layout, fht_quadrant q, int64_t in_pitch,
                            void *grad_img, int64_t img_batch_stride, int64_t out_pitch,
                            void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------ batched
 * Many images of different sizes in one persistent launch. Each image is
 * transformed exactly as fht_forward would transform it (same quadrant and
 * types for the whole batch), padded to its own power of two; the launch takes
 * work items of all images from one queue, ordered by pass, and an item of a
 * later pass waits for its image's previous pass (the waits are bounded; see
 * fht_batched_status). Not in the paper: batching is how the library runs many
 * small transforms at once. Supported: uint8 -> int32 and float32 -> float32,
 * images up to 4096 padded rows (4096 padded columns for Q2/Q3). */
typedef struct fht_plan fht_plan;   /* opaque, host-side */

typedef struct {
    const void *img;     /* DEVICE pointer to image j, h_j x w_j, pitch img_pitch */
    int64_t img_pitch;   /* elements, >= w_j */
    void *out;           /* DEVICE pointer to its quadrant, n_j x W_j, pitch out_pitch */
    int64_t out_pitch;   /* elements, >= W_j (fht_query_shape) */
} fht_image_desc;

/* Plan a batch of `count` images with sizes hs[j] x ws[j] (HOST arrays).
 * Writes the plan (free with fht_plan_destroy) and the device workspace it
 * needs (intermediate levels of every image, the work tables and counters;
 * for float32 plans enough for fht_adjoint_batched as well). Allocates only
 * host memory (pinned staging for the tables). */
fht_status fht_plan_create_batched(const int *hs, const int *ws, int count, fht_quadrant q,
                                   fht_dtype in_t, fht_dtype acc_t, fht_plan **plan,
                                   size_t *workspace_bytes);

/* How batched plans cut their work (not in the paper; every setting gives the
 * same results bit for bit). Read when a plan is created; the package's
 * autotuner times the candidates on a batch and sets the fastest. */
typedef struct {
    int units_per_item;   /* (group, tile) units one claimed work item covers:
                             the per-item bookkeeping is paid once for them;
                             1..16 (default 4) */
    int tile_u8;          /* warp-widths (248 columns) of block-A source columns
                             in first passes over uint8 images: 1..3 (default 2) */
    int tile_wide;        /* the same for passes with 4-byte shared tiles: 1..3
                             (default 1, widened to one block-A item per warp) */
    int ctas_per_sm;      /* CTAs of the persistent kernel per SM, i.e. its
                             register budget: 2 (128 registers) or 3 (80);
                             default 2 */
    int first_levels[13]; /* index K (7..12): butterfly levels of the first of
                             the two passes of an image with 2^K padded rows
                             ("stages per CTA"), K-6..6; 0 = the default
                             ceil(K/2). Entries below 7 are ignored (images
                             up to 64 rows take one pass). */
} fht_batched_tuning;

/* Use `t` for batched plans created from now on, process-wide; NULL restores
 * the defaults. FHT_EINVAL for values out of range (nothing changes). */
fht_status fht_set_batched_tuning(const fht_batched_tuning *t);

/* The batched tuning in use (HOST struct). */
fht_status fht_get_batched_tuning(fht_batched_tuning *out);

/* Transform the batch: descs is a HOST array of `count` descriptors, checked
 * against the plan; workspace is >= workspace_bytes, 256-byte aligned. One
 * host-to-device copy of the tables, one memset and one kernel launch on
 * `stream`, all capturable in a CUDA graph. The descriptors are staged in
 * pinned host memory owned by the plan: three tables used in turn by direct
 * calls (a call first waits until the copy of the call that used its table
 * last has run), and one more table for every stream capture, allocated by
 * the capturing call and kept until fht_plan_destroy, so that each graph
 * replays the descriptors given when it was captured, whatever the plan runs
 * or captures later (each capture holds a few hundred bytes per pass of every
 * image; FHT_ENOMEM if that table cannot be allocated). A plan serves one
 * stream at a time. */
fht_status fht_forward_batched(fht_plan *plan, const fht_image_desc *descs, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Per-image arguments of fht_adjoint_batched. */
typedef struct {
    const void *grad_hough;     /* DEVICE pointer: gradient w.r.t. quadrant j, n_j x W_j
                                   float32, read only */
    int64_t grad_hough_pitch;   /* elements, >= W_j (fht_query_shape) */
    void *grad_img;             /* DEVICE pointer: gradient w.r.t. image j, h_j x w_j
                                   float32, fully overwritten */
    int64_t grad_img_pitch;     /* elements, >= w_j */
} fht_adjoint_desc;

/* Adjoint of the batch (float32 plans only; FHT_EUNSUPPORTED otherwise):
 * for every image j, grad_img = H_j^T grad_hough, the transpose of its
 * quadrant transform, exactly (bit for bit) what fht_adjoint with layout
 * FHT_LAYOUT_QUADRANT and the plan's quadrant computes. Not in the paper: the
 * transform is linear and the back-projection is its transpose, used by
 * gradient-based reconstruction over many images of different sizes. One
 * persistent launch as fht_forward_batched (same staging, capture and status
 * rules; descs is a HOST array of `count` descriptors, workspace >= the
 * plan's workspace_bytes, 256-byte aligned, shared with the forward calls of
 * the same stream). */
fht_status fht_adjoint_batched(fht_plan *plan, const fht_adjoint_desc *descs, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Wait for `stream` and report the last batched launch's device status in
 * `workspace`: FHT_OK, or FHT_ETIMEOUT if a pass dependency wait exceeded
 * its budget (the affected items were skipped and the launch still ended). */
fht_status fht_batched_status(const fht_plan *plan, const void *workspace, void *stream);

/* Test hook: the clock budget (SM cycles) of each dependency wait, and a
 * number added to every dependency target (dep_bias > 0 makes the waits
 * unsatisfiable, so that tests can check the timeout path). */
fht_status fht_batched_test_hooks(fht_plan *plan, long long wait_budget_cycles, int dep_bias);

void fht_plan_destroy(fht_plan *plan);

/* Device status of the transforms' kernels. Waits for every launch issued so
 * far in this process, then returns FHT_EBOUNDS if a kernel of the debug
 * build refused an access since the last call (the count is then reset),
 * else FHT_OK; FHT_ECUDA if the device could not be synchronised. The debug
 * build (compiled with -DFHT_DEBUG, see below) checks every global load and
 * store of the pass kernels against the buffers the pass may touch and skips
 * (a load reads zero) and counts any access outside them; the release
 * build's kernels check nothing, so there the status is FHT_OK whenever the
 * device synchronises. Not in the paper. */
fht_status fht_device_status(void);

/* Test hook of the debug build's bounds checks: every pass launched from now
 * on records a destination span `shrink_bytes` shorter than its buffer, so
 * that its last stores are refused (and skipped) and fht_device_status
 * reports FHT_EBOUNDS; 0 restores the exact spans. Nothing outside the
 * buffers is ever touched. FHT_EUNSUPPORTED in the release build, FHT_EINVAL
 * for a negative value. */
fht_status fht_debug_test_hooks(long long shrink_bytes);

/* ------------------------------------------------------------ tuning
 * How the plain sum transforms and adjoints (fht_forward, fht_forward_range,
 * fht_full_quadrants, fht_adjoint, the uniform batches, fht_forward_static)
 * of quadrants with n = 2^K rows are split into fused passes and tiled. Not
 * in the paper (it fixes what is computed, not how the work is cut); every
 * setting gives the same results bit for bit. The package's autotuner times
 * the candidates on the GPU and sets the fastest per K. */
typedef struct {
    int max_levels;   /* most butterfly levels one pass fuses ("stages per
                         CTA"): 4, 5 or 6; the K levels are split into
                         ceil(K / max_levels) passes as evenly as possible */
    int tile_u8;      /* warp-widths (248 columns each) of source columns per
                         tile in first passes over uint8 images: 1, 2 or 3 */
    int tile_wide;    /* the same for passes with 4-byte shared tiles: 1..3 */
} fht_tuning;

/* Use `t` for quadrants with 2^K rows (1 <= K <= 15) in calls made from now
 * on, process-wide (a CUDA graph keeps the plan it captured). Workspace sizes
 * follow the tuning: query fht_workspace_size after setting it (a call whose
 * workspace is too small for its plan returns FHT_EINVAL). t == NULL restores
 * the default (6 levels; tile widths 1, or those of FHT_TUNE="a,b" in the
 * environment when the library loads). FHT_EINVAL for K or values out of
 * range. */
fht_status fht_set_tuning(int K, const fht_tuning *t);

/* The tuning in use for quadrants with 2^K rows (HOST struct). */
fht_status fht_get_tuning(int K, fht_tuning *out);

/* ------------------------------------------------------------ profiling
 * Kernel-level timing for benchmarks; normal use never needs it. Not in the
 * paper. While profiling is on, every kernel launch made by this library is
 * bracketed by a pair of CUDA events recorded on the launch's own stream;
 * fht_profile_end waits for those events and returns, per kernel name, the
 * number of launches and their summed device time. */
typedef struct {
    char name[64];
    int launches;
    double total_ms;
    double alg_bytes;   /* summed algorithmic bytes of those launches: the level
                           each reads as stored plus the level it writes */
} fht_kernel_time;

/* Start (or restart) recording; previous records are dropped. */
fht_status fht_profile_begin(void);

/* Stop recording, synchronize the recorded events and write up to `capacity`
 * per-kernel totals (HOST array) to `out`; *count receives the number of
 * distinct kernel names seen (may exceed capacity). Profiling is process-wide
 * and not meant for use during stream capture. */
fht_status fht_profile_end(fht_kernel_time *out, int capacity, int *count);

/* Number of kernel launches this library has issued since it was loaded. */
long long fht_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* FHT_H */
