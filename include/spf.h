/*
 * spf.h -- C ABI of the GB300 M-TIP slice / match / merge library.
 *
 * The library computes the data-parallel path of the Cartesian-NUFFT M-TIP
 * reconstruction (arXiv 2109.05339, Sec. II): slicing a 3D model with a
 * type-2 NUFFT (Sec. II-A), matching every experimental image to its nearest
 * model image (Sec. II-B), and merging the oriented images through the
 * Tikhonov normal equations of Eq. 2 solved by conjugate gradient on the
 * Toeplitz form of A*DA (Sec. II-C).
 *
 * Conventions shared by every call
 *   - Model grid: N odd, modes n in {-M..M}^3, M = (N-1)/2, stored as float
 *     [n_z+M][n_y+M][n_x+M] (x fastest), N^3 values.
 *   - q-points: the NUFFT coordinate of a physical q is t = 2 pi dr q with
 *     dr = 1/(N dq), dq = qmax/M, so grid point q = m dq has t = 2 pi m / N.
 *   - Quaternions: 4 floats (w, x, y, z) per orientation, unit norm, active
 *     rotation; a detector point q_lab[p] is rotated to R(quat) q_lab[p].
 *   - q_lab: 3 floats (x, y, z) per detector pixel, P2 pixels.
 *   - Images / slices: row-major [orientation or image][pixel], float.
 *   - Every array pointer is a DEVICE pointer owned by the caller unless the
 *     argument says "host". The library never frees caller memory.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) unless it says otherwise, and returns an int
 *     status: SPF_OK or a negative SPF_ERR_* code. spf_last_error_string()
 *     gives a message for the last failure on the calling thread.
 *   - A plan or matcher is used by one stream at a time and is not thread
 *     safe; after any error it stays usable.
 *   - No call allocates device memory except the *_create functions and
 *     spf_mtip_set_orientations (which creates point sets).
 */
#ifndef SPF_H
#define SPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPF_OK 0
#define SPF_ERR_ARG (-1)         /* bad argument (size, pointer, limit)          */
#define SPF_ERR_OOM (-2)         /* device allocation failed at create           */
#define SPF_ERR_CUDA (-3)        /* a CUDA runtime call or launch failed         */
#define SPF_ERR_TIMEOUT (-4)     /* a bounded device wait gave up                */
#define SPF_ERR_UNSUPPORTED (-5) /* option not built for this device             */

#define SPF_FP32 0 /* cross term in FP32 on the CUDA cores                      */
#define SPF_BF16 1 /* cross term in BF16 on the tensor cores, FP32 accumulate  */
#define SPF_FP8 2  /* cross term in FP8 e4m3 with per-row scales, FP32 acc.   */

#define SPF_MAX_TOPK 8

typedef struct spf_plan spf_plan;
typedef struct spf_matcher spf_matcher;

/* Message for the last failing call on this thread ("" if none). Host. */
const char* spf_last_error_string(void);

/* Library ABI version (increments on any signature change). Host. */
int spf_version(void);

/* ---------------------------------------------------------------------------
 * NUFFT plan (Sec. II-A and II-C: type-2 slicing, type-1 merging).
 *
 * N         model grid side (odd, 3..1023).
 * qmax      largest |q| of the model grid (> 0).
 * eps       NUFFT tolerance (1e-7 .. 1e-2); sets the exponential-of-semicircle
 *           kernel width w = ceil(log10(1/eps)) + 1 and shape beta = 2.3 w,
 *           with upsampling 2.
 * max_points  the most nonuniform points one type-1 call may pass (images x
 *           pixels), < 2^31; sizes the point-sort buffer. Type-2 calls sort
 *           and interpolate in chunks of whole orientations of at most this
 *           many points (unsorted if not even one orientation fits).
 * device    CUDA device ordinal; the plan allocates its scratch there.
 * Allocates the fine grids (n_f^3 for N modes, n_fT^3 for the 2N-1 modes of
 * the Toeplitz kernel, P_T^3 for the circulant embedding), a sort buffer of
 * 4 * max_points bytes, per-cell sort counters (about 12 bytes per fine cell
 * of each grid), and the CG vectors. Synchronous. *out owns them.
 * ------------------------------------------------------------------------- */
int spf_plan_create(spf_plan** out, int N, double qmax, double eps, int64_t max_points,
                    int device);
int spf_plan_destroy(spf_plan* plan);

/* Device-side error word of the plan (bounds checks inside kernels): waits
 * for the device (cudaDeviceSynchronize on the plan's device), returns SPF_OK
 * or SPF_ERR_ARG if a kernel found an inconsistent point, then clears it. */
int spf_plan_status(spf_plan* plan);

/* Sizes chosen by the plan (host): fine grid n_f, Toeplitz fine grid n_fT,
 * embedding P_T, kernel width w. Any pointer may be NULL. */
int spf_plan_sizes(const spf_plan* plan, int* nf, int* nfT, int* PT, int* w);

/* Slicing, Sec. II-A: the type-2 NUFFT of the model at rotated detector points.
 *   slices[j*P2 + p] = Re sum_n A[n] exp(-i n . t_jp),
 *   t_jp = 2 pi dr R(quats[j]) q_lab[p],   j < M, p < P2.
 * A: N^3 floats (only its even part contributes to the real part).
 * quats: M x 4, q_lab: P2 x 3, slices: M x P2 (written). M*P2 < 2^32. */
int spf_slice_model(spf_plan* plan, const float* A, const float* quats, int M,
                    const float* q_lab, int P2, float* slices, void* stream);

/* Adjoint of spf_slice_model (Sec. II-C type 1), the backward of slicing:
 *   gradA[n] (+)= Re sum_{j,p} g[j*P2 + p] exp(+i n . t_jp).
 * accumulate = 0 overwrites gradA, 1 adds to it. M*P2 <= max_points. */
int spf_slice_adjoint(spf_plan* plan, const float* g, const float* quats, int M,
                      const float* q_lab, int P2, float* gradA, int accumulate,
                      void* stream);

/* Type-2 / type-1 at explicit points t (npts x 3 floats, radians, any real
 * value; taken mod 2 pi). type2: out[j] = Re sum_n A[n] exp(-i n.t_j).
 * type1: out[n] (+)= Re sum_j v[j] exp(+i n.t_j), npts <= max_points. */
int spf_nufft_type2(spf_plan* plan, const float* A, const float* pts, int64_t npts,
                    float* out, void* stream);
int spf_nufft_type1(spf_plan* plan, const float* v, const float* pts, int64_t npts,
                    float* out, int accumulate, void* stream);

/* ---------------------------------------------------------------------------
 * Point sets: the rotated detector points of a fixed orientation set, sorted
 * once for both fine grids (the "set points" step of a NUFFT plan). The paper
 * slices at "a predetermined set of orientations" (Sec. II-A) that does not
 * change between M-TIP iterations, so slicing and merging reuse the sort.
 *
 * spf_points_create: copies quats (M x 4) and q_lab (P2 x 3) and sorts the
 *   M*P2 points (M*P2 < 2^31). Allocates about 16 bytes per point (a sort
 *   order for each grid, the inverse of the model-grid order, class sums) --
 *   a create call. Stream-ordered after the copies. flags: 0, or
 *   SPF_POINTS_SLICE_ONLY to sort for slicing alone (4 bytes per point; such a
 *   set cannot merge: spf_merge_points returns SPF_ERR_ARG).
 * spf_slice_points: as spf_slice_model for the set's orientations;
 *   slices: M x P2.
 * spf_merge_points: Sec. II-C merge by class sums. Images whose orientation
 *   orient_idx[i] falls in [orient_offset, orient_offset + M) are summed per
 *   orientation (weighted by D[p] b_scale) -- the class sums of the M-TIP
 *   pipeline -- and the class sums and class counts are spread at the set's
 *   points. By linearity the result equals spf_merge_images with
 *   quats[orient_idx[i]] for those images:
 *     rhs        (+)= Re sum_{j,p} (sum_{i in class j} D[p] b_scale img[i,p]) e^{+i n.t_jp}
 *     kernel_hat (+)= FFT_{P_T}(embed Re sum_{j,p} count_j D[p] e^{+i d.t_jp}).
 *   Images outside the range are ignored (chunked orientation sets add up
 *   with accumulate = 1). Either output may be NULL.
 * ------------------------------------------------------------------------- */
typedef struct spf_points spf_points;
#define SPF_POINTS_SLICE_ONLY 1
int spf_points_create(spf_points** out, spf_plan* plan, const float* quats, int M, const float* q_lab,
                      int P2, int flags, void* stream);
int spf_points_destroy(spf_points* pts);
int spf_slice_points(spf_plan* plan, spf_points* pts, const float* A, float* slices, void* stream);
int spf_merge_points(spf_plan* plan, spf_points* pts, const float* images, const int32_t* orient_idx,
                     int n_img, int orient_offset, const float* D, float b_scale, float* rhs,
                     float* kernel_hat, int accumulate, void* stream);

/* ---------------------------------------------------------------------------
 * Deferred merge over many chunks (Sec. II-C). The type-1 sums are linear,
 * so the chunks' spread fine grids add up before any transform: the
 * right-hand side and the Toeplitz kernel are transformed once, however many
 * orientation or image chunks feed them (the kernel is "computed just once").
 * spf_merge_begin: clears the plan's two fine grids and opens the merge.
 * spf_merge_points_add: spf_merge_points for one point set, spreading onto
 *   the open merge instead of producing rhs / kernel_hat; want_rhs and
 *   want_kernel (0 / 1) select the sums.
 * spf_merge_images_add: spf_merge_images likewise.
 * spf_merge_finish: transforms the grids and closes the merge:
 *   rhs (+)= the right-hand side, kernel_hat (+)= the kernel spectrum, exactly
 *   as the single-call forms give them for all chunks together; either may
 *   be NULL (its sum is dropped).
 * While a merge is open, calls that write the fine grids (slicing, type-1,
 * the single-call merges) return SPF_ERR_ARG; *_add and finish without an
 * open merge return SPF_ERR_ARG. Stream-ordered like the other calls.
 * ------------------------------------------------------------------------- */
int spf_merge_begin(spf_plan* plan, void* stream);
int spf_merge_points_add(spf_plan* plan, spf_points* pts, const float* images, const int32_t* orient_idx,
                         int n_img, int orient_offset, const float* D, float b_scale, int want_rhs,
                         int want_kernel, void* stream);
int spf_merge_images_add(spf_plan* plan, const float* images, const float* quats, int n_quats,
                         const int32_t* orient_idx, int n_img, const float* q_lab, int P2, const float* D,
                         float b_scale, int want_rhs, int want_kernel, void* stream);
int spf_merge_finish(spf_plan* plan, float* rhs, float* kernel_hat, int accumulate, void* stream);

/* ---------------------------------------------------------------------------
 * Merge, Sec. II-C (Eq. 2 with the Toeplitz method): from one chunk of
 * oriented images build
 *   rhs[n]        (+)= Re sum_{i,p} D[p] b_scale images[i*P2+p] exp(+i n.t_ip)
 *   kernel_hat[k] (+)= FFT_{P_T}( embed K )[k],
 *        K(d) = Re sum_{i,p} D[p] exp(+i d.t_ip),  d in {-(N-1)..N-1}^3,
 * t_ip from the orientation of image i and q_lab[p]: quats[orient_idx[i]] when
 * orient_idx (n_img int32, e.g. the matcher's best indices) is given, else
 * quats[i]; quats holds n_quats rows. An index outside [0, n_quats) sets the
 * plan's error word (spf_plan_status) and is clamped.
 * K is embedded circulantly in P_T^3 (P_T = smallest even 2/3/5-smooth
 * >= 2N-1); kernel_hat is real, P_T^3 floats, layout [z][y][x].
 * D: P2 per-pixel weights (1 valid, 0 masked) or NULL for all ones.
 * Linear in the images: chunks are summed with accumulate = 1 (the paper's
 * per-node type-1 NUFFTs followed by a sum reduction).
 * n_img*P2 <= max_points. */
int spf_merge_images(spf_plan* plan, const float* images, const float* quats, int n_quats,
                     const int32_t* orient_idx, int n_img, const float* q_lab, int P2,
                     const float* D, float b_scale, float* rhs, float* kernel_hat, int accumulate,
                     void* stream);

/* Conjugate gradient on H x = rhs + lambda x0, H = Re(A^H D A) + lambda I
 * applied as crop(IFFT(kernel_hat * FFT(pad x))) + lambda x (Eq. 2, Sec. II-C).
 * spf_cg_begin: x = x0, r = rhs + lambda x0 - H x0, p = r (state in the plan).
 * spf_cg_merge_step: one CG iteration updating x in place. The step length
 * and direction update are computed on the device from FP64 inner products;
 * no host synchronisation. res_norm (device, may be NULL) receives |r| after
 * the step as a double. x, rhs, x0: N^3 floats; kernel_hat: P_T^3 floats. */
int spf_cg_begin(spf_plan* plan, const float* kernel_hat, double lambda, const float* rhs,
                 const float* x0, float* x, double* res_norm, void* stream);
int spf_cg_merge_step(spf_plan* plan, const float* kernel_hat, double lambda, float* x,
                      double* res_norm, void* stream);

/* L-curve quantities of a merge solution x (Sec. II-C: the regularisation
 * parameter is chosen on the L-curve). out (device, 2 doubles):
 *   out[0] = |A x - b|_D^2 = x.T x - 2 x.rhs + b_norm2[0]
 *   out[1] = |x - x0|^2
 * with T x the Toeplitz product without lambda, rhs the merge right-hand side
 * Re(A^H D b) and b_norm2 (device, 1 double, may be NULL for 0) = b.D b from
 * spf_weighted_sumsq. FP64 reductions; uses the plan's CG scratch, so call it
 * between CG solves, not inside one. */
int spf_cg_objective(spf_plan* plan, const float* kernel_hat, const float* rhs, const float* x,
                     const float* x0, const double* b_norm2, double* out, void* stream);
/* L-curve corner (host; Sec. II-C): for a sweep of n >= 3 increasing
 * lambdas with res2[k] = |A x_k - b|_D^2 and reg2[k] = |x_k - x0|^2 (all
 * positive; host arrays, e.g. copied back from spf_cg_objective), *index is
 * the interior point of maximum curvature of (log |A x - b|_D, log |x - x0|)
 * as functions of log lambda (three-point derivatives on the uneven grid);
 * kappa (host, n - 2 doubles, may be NULL) receives the curvature at the
 * interior points 1 .. n - 2. */
int spf_lcurve_corner(const double* lams, const double* res2, const double* reg2, int n, int* index,
                      double* kappa);
/* out[0] (+)= sum_{i,p} D[p] (scale images[i*P2+p])^2 in FP64 (D NULL: ones). */
int spf_weighted_sumsq(spf_plan* plan, const float* images, int n_img, int P2, const float* D,
                       float scale, double* out, int accumulate, void* stream);

/* Gradient-based merge (the differentiation pattern of slicing): with S_i
 * the slice at image i's orientation (Sec. II-A) and S^T its type-1 adjoint
 * (Sec. II-C),
 *   L(x) = 1/2 sum_{i,p} D[p] (S_i x - b_scale images[i*P2+p])^2 + lambda/2 |x - x0|^2,
 *   grad = S^T D (S x - b_scale images) + lambda (x - x0).
 * For x even in n, S^T D S = Re(A^H D A): L is the objective of Eq. 2.
 * Slices are recomputed chunk by chunk (chunk images at a time, chunk * P2 <=
 * max_points) into `work` (chunk * P2 floats, caller-owned), never stored.
 * quats: n_img x 4 (image i's orientation), images: n_img x P2, D: P2 or NULL.
 * spf_slice_loss_grad: *loss (device double) = L(x), grad (N^3) = grad L(x);
 *   x0 may be NULL when lambda = 0.
 * spf_slice_normal_apply: out = S^T D S v + lambda v (N^3).
 * spf_gradient_step: one steepest-descent step with exact line search on the
 *   quadratic L: *loss = L(x) before the step, grad and Hg (N^3 work, written)
 *   = g and H g with H = S^T D S + lambda I, then x -= (g.g / g.Hg) g (no step
 *   when g.Hg <= 0 or g = 0). Inner products FP64, step length on the device.
 * All three use the plan's fine grids (refused while a deferred merge is
 * open) and reduction scratch; FP64 loss and inner products. */
int spf_slice_loss_grad(spf_plan* plan, const float* x, const float* x0, const float* quats, int n_img,
                        const float* q_lab, int P2, const float* images, float b_scale, const float* D,
                        double lambda, int chunk, float* work, double* loss, float* grad, void* stream);
int spf_slice_normal_apply(spf_plan* plan, const float* v, const float* quats, int n_img, const float* q_lab,
                           int P2, const float* D, double lambda, int chunk, float* work, float* out,
                           void* stream);
int spf_gradient_step(spf_plan* plan, float* x, const float* x0, const float* quats, int n_img,
                      const float* q_lab, int P2, const float* images, float b_scale, const float* D,
                      double lambda, int chunk, float* work, float* grad, float* Hg, double* loss,
                      void* stream);

/* H x without the CG state (Toeplitz form): out = crop(IFFT(kernel_hat *
 * FFT(pad x))) + lambda x. Used to check the operator. */
int spf_toeplitz_apply(spf_plan* plan, const float* kernel_hat, double lambda,
                       const float* x, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Orientation matching, Sec. II-B: for every image the model image nearest in
 * Euclidean distance d_ij = |x_i|^2 + |y_j|^2 - 2 x_i . y_j (x_i = img_scale *
 * image i). The cross term runs in `precision`; with BF16 and FP8 the norms
 * are those of the quantised rows, so the approximate distance is the distance
 * between the quantised image and model image (0 for an image equal to a model
 * image). The best `topk` candidates per image by that distance are then
 * re-ranked with exact FP32 distances sum_p (x_ip - y_jp)^2,
 * so the returned argmin and distances are FP32-exact over the candidates.
 * Ties go to the lower orientation index. Model images can be streamed in
 * chunks: orient_offset is added to the indices of each chunk, and the
 * running best-topk list per image survives across calls.
 *
 * spf_matcher_create: max_images, max_orient_chunk bound later calls; P2 is
 *   fixed; precision SPF_FP32 / SPF_BF16 / SPF_FP8; 2 <= topk <= 8.
 *   Allocates quantised copies and candidate buffers. Synchronous.
 * spf_matcher_set_images: computes norms and quantised copies of the images
 *   and resets the running lists. images: n_img x P2 floats; the matcher keeps
 *   the pointer, which must stay valid until the last add_slices.
 * spf_matcher_add_slices: matches one chunk of n_orient model images
 *   (n_orient x P2 floats, valid until the call's work completes).
 * spf_matcher_results: best_idx, best_d, second_d: n_img each (may be NULL);
 *   topk_idx, topk_d: n_img x topk (may be NULL). Distances are in the units
 *   of img_scale * images.
 * ------------------------------------------------------------------------- */
int spf_matcher_create(spf_matcher** out, int max_images, int max_orient_chunk, int P2,
                       int precision, int topk, int device);
int spf_matcher_destroy(spf_matcher* m);
/* Device-side error word of the matcher: waits for the device, returns SPF_OK,
 * SPF_ERR_TIMEOUT (a bounded pipeline wait in a tensor-core kernel gave up;
 * its results are not valid) or SPF_ERR_CUDA (tensor memory could not be
 * allocated), then clears it. */
int spf_matcher_status(spf_matcher* m);
int spf_matcher_set_images(spf_matcher* m, const float* images, int n_img, float img_scale,
                           void* stream);
/* The same for images given as 16-bit photon counts (n_img x P2 uint16,
 * device, 8-byte aligned rows read as vectors when P2 % 4 == 0): the
 * quantised copies and the FP32 re-rank read the counts themselves (exact in
 * FP32), so no FP32 copy is needed. BF16 and FP8 matchers only
 * (SPF_ERR_UNSUPPORTED for SPF_FP32, whose CUDA-core path reads FP32 rows). */
int spf_matcher_set_images_u16(spf_matcher* m, const uint16_t* images, int n_img, float img_scale,
                               void* stream);
/* Pixel weights for the distance, d_ij = sum_p D[p] (x_ip - y_jp)^2 (D >= 0;
 * D = 0 excludes a pixel, e.g. behind the beam stop of Sec. II-C). D: P2
 * floats (device) or NULL for all ones. Takes effect for the next
 * set_images / add_slices calls: set it before set_images. */
int spf_matcher_set_mask(spf_matcher* m, const float* D, void* stream);
int spf_matcher_add_slices(spf_matcher* m, const float* slices, int n_orient,
                           int orient_offset, void* stream);
/* Tile schedule of the tensor-core cross term (BF16 / FP8; host, takes effect
 * at the next add_slices): 0 (default) lets a model of tensor-core time and
 * HBM traffic choose, 1 forces contiguous ranges of the image-major tile
 * order, 2 forces a grid of CTAs over image-tile x orientation-tile ranges
 * (concurrent CTAs share operand tiles; the model's choice for many image
 * tiles). The results differ only in which approximate candidates tie. */
int spf_matcher_set_schedule(spf_matcher* m, int schedule);
/* When the exact re-rank runs (host; set before spf_matcher_set_images).
 * deferred = 0 (default): each add_slices call re-ranks its own best
 * candidates, so its slices are needed only until its work completes.
 * deferred = 1: every call merges its candidates into a running approximate
 * top-8 per image, and the exact FP32 re-rank of that list runs once, in
 * spf_matcher_results, reading each image once. The slices of every
 * add_slices call since set_images must then stay valid and unchanged until
 * spf_matcher_results; calls must cover increasing, non-overlapping
 * orientation ranges (at most 1024 of them). The re-ranked candidates are
 * the best 8 by approximate distance over all chunks, instead of the best 8
 * of each chunk. */
int spf_matcher_set_rerank(spf_matcher* m, int deferred);
int spf_matcher_results(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                        int32_t* topk_idx, float* topk_d, void* stream);

/* One-shot Sec. II-B matching of n_img images against n_orient model images
 * with the matcher's buffers: set_images, add_slices (offset 0), results.
 * best_idx, best_d, second_d: n_img each (device). */
int spf_match_orientations(spf_matcher* m, const float* images, int n_img, float img_scale,
                           const float* slices, int n_orient, int32_t* best_idx,
                           float* best_d, float* second_d, void* stream);

/* ---------------------------------------------------------------------------
 * M-TIP iteration driver (Fig. 3 without phasing; Sec. II-A to II-C): the
 * slice -> match -> merge -> CG iteration over a fixed orientation set,
 * orchestrated in the library.
 *
 * The orientation set is the run's configuration ("a predetermined set of
 * orientations", Sec. II-A): spf_mtip_set_orientations takes it once and the
 * driver renumbers it along a Morton curve of the quaternions (neighbouring
 * indices are neighbours on SO(3), which keeps candidate model images of
 * images re-ranked together in L2). Its points are either sorted per
 * orientation chunk once and kept (about 16 bytes per orientation x pixel);
 * or only their sort for slicing is kept (about 4 bytes per orientation x
 * pixel) while the merge spreads image chunks at their matched orientations;
 * or, beyond that budget too, they are re-sorted per chunk for slicing on
 * every iteration and the merge spreads image chunks. Orientation indices passed in or out are in the caller's
 * numbering; exact distance ties resolve to the lower index in the driver's.
 *
 * An iteration (spf_mtip_iteration): (1) the model A is sliced at every
 * orientation chunk and every image is matched against each chunk (running
 * top-k with the FP32 re-rank); (2) the images are merged at their best
 * orientations -- every chunk spread onto the plan's fine grids, transformed
 * once into the right-hand side and the Toeplitz kernel; (3) cg_iters CG
 * steps on Eq. 2 from x0 = A, lambda = lam_rel * (sum of the pixel weights
 * over all merged images). The three steps are also separate calls, so that
 * image-sharded processes can add their right-hand sides and kernels between
 * merge and solve.
 *
 * Images are FP32 (SPF_IMAGES_F32) or unsigned 16-bit photon counts
 * (SPF_IMAGES_U16, converted to FP32 on the device inside the call).
 *
 * spf_mtip_config: N, qmax, eps as spf_plan_create; P2 pixels; max_images
 *   per call; n_orient orientations; orient_chunk orientations sliced and
 *   matched per chunk (0: all); img_chunk images merged per type-1 pass when
 *   streaming (0: all); precision and topk as spf_matcher_create;
 *   cache_points 1 keep the sorted point sets, 2 keep slice-only sets and
 *   merge image chunks, 0 stream (re-sort per chunk, merge image chunks),
 *   -1 choose: 1 when 16 * n_orient * P2 bytes fit point_budget_bytes (<= 0:
 *   half of the device's free memory at create), else 2 when 4 * n_orient *
 *   P2 bytes do, else 0; host_image_type SPF_IMAGES_F32 /
 *   SPF_IMAGES_U16 allocates two device input slots for
 *   spf_mtip_iteration_host, -1 none; device ordinal.
 * spf_mtip_create allocates the plan, the matcher, a slice chunk, an FP32
 *   image buffer (max_images x P2), the merge and CG buffers and the host-path
 *   slots. Synchronous. spf_mtip_set_orientations copies quats (n_orient x 4)
 *   and q_lab (P2 x 3) and, when keeping point sets (full or slice-only),
 *   creates and sorts them (it allocates: a set-up call); synchronous. spf_mtip_set_mask: pixel
 *   weights D (P2 floats, device, >= 0, caller-owned and kept until replaced)
 *   for matching, merging and lambda, or NULL for ones; synchronous.
 * spf_mtip_match: best (n_img, device) in the caller's numbering; best_d,
 *   second_d (n_img) and topk_idx, topk_d (n_img x topk) optional (NULL).
 * spf_mtip_merge: right-hand side (N^3) and kernel spectrum (P_T^3) of the
 *   images at orientations best (caller's numbering) into rhs, kernel_hat
 *   (device, caller-owned, overwritten).
 * spf_mtip_solve: CG from x0 for cg_iters steps into x (N^3), lambda =
 *   lam_rel * (sum of D over a pixel row) * n_img_total; *lambda_out (host,
 *   may be NULL) receives it; res_hist (device, cg_iters + 1 doubles, may be
 *   NULL) the residual norms.
 * spf_mtip_iteration: the three steps; best (device, may be NULL) and x
 *   (device) are written.
 * spf_mtip_iteration_host: the same from and to HOST buffers: A_host (N^3
 *   floats) and images_host (n_img x P2 of host_image_type) are copied into
 *   one of two device slots on the driver's own copy stream, which waits until
 *   the call two back is done with that slot, so that a call's copies overlap
 *   the previous call's compute; best_host (n_img int32) and x_host (N^3
 *   floats) are written back on `stream`. Asynchronous for page-locked host
 *   buffers: the inputs must stay unchanged and the outputs are valid once
 *   `stream` has completed the call's work (e.g. cudaStreamSynchronize).
 * spf_mtip_upload_host / spf_mtip_release_upload: the upload half of
 *   spf_mtip_iteration_host for callers that run the steps themselves (an
 *   image-sharded run whose merge sums are reduced across processes between
 *   merge and solve, Sec. II-C). upload_host copies A_host and images_host
 *   into the next device slot exactly as the iteration does and returns the
 *   slot's device pointers (A_dev: N^3 floats, images_dev: n_img x P2 of
 *   host_image_type), valid for work enqueued on `stream`; release_upload
 *   marks the slot free once the work enqueued on `stream` so far completes.
 *   One upload is held at a time (SPF_ERR_ARG for a second before release).
 * spf_mtip_set_upload: how spf_mtip_iteration_host moves the images to the
 *   device. SPF_UPLOAD_SM (default): a kernel on the copy stream reads the
 *   host buffer over the CPU-GPU link and writes the slot (about 190 GB/s on
 *   a GB300 while the previous call computes, against 35-45 GB/s for the
 *   copy engines there); taken only when the first and last byte of
 *   images_host lie in page-locked memory mapped into the device's address
 *   space (cudaHostAlloc / cudaHostRegister, one allocation for the whole
 *   buffer) and both ends are 16-byte aligned, else the copy engines are
 *   used. SPF_UPLOAD_COPY: always cudaMemcpyAsync on the copy stream (no SMs
 *   taken from the computing call). SPF_ERR_ARG for another mode.
 * spf_mtip_last_upload_ms: device time of the most recent completed image
 *   upload of spf_mtip_iteration_host (events around it on the copy stream);
 *   -1 before the first. Waits for that upload to finish.
 * spf_mtip_status: the plan's, the matcher's and the driver's error words
 *   (waits for the device). spf_mtip_plan / spf_mtip_matcher: the driver's
 *   plan and matcher (owned by the driver) for the other calls of this header.
 * spf_mtip_info: the point-set mode in use (cache_points: 1 full sets kept,
 *   2 slice-only sets kept, 0 streamed), the chunk sizes in use, and whether
 *   all slices are kept (one deferred re-rank per iteration).
 * ------------------------------------------------------------------------- */
#define SPF_IMAGES_F32 0
#define SPF_IMAGES_U16 1
#define SPF_UPLOAD_COPY 0
#define SPF_UPLOAD_SM 1
typedef struct spf_mtip spf_mtip;
typedef struct spf_mtip_config {
  int N;
  double qmax;
  double eps;
  int P2;
  int max_images;
  int n_orient;
  int orient_chunk;
  int img_chunk;
  int precision;
  int topk;
  int cache_points;
  int64_t point_budget_bytes;
  int host_image_type;
  int device;
  int keep_slices;
} spf_mtip_config;
/* The driver's renumbering of an orientation set (host; no device work):
 * order_host[i] = the caller's index of driver index i, the permutation that
 * sorts the Morton codes of the quaternions' (x, y, z), each quantised to 10
 * bits over [-1, 1] (stable for equal codes). quats_host: M x 4 floats. */
int spf_morton_order(const float* quats_host, int M, int32_t* order_host);
int spf_mtip_create(spf_mtip** out, const spf_mtip_config* cfg);
int spf_mtip_destroy(spf_mtip* h);
int spf_mtip_info(const spf_mtip* h, int* cache_points, int* orient_chunk, int* img_chunk, int* keep_slices);
spf_plan* spf_mtip_plan(spf_mtip* h);
spf_matcher* spf_mtip_matcher(spf_mtip* h);
int spf_mtip_status(spf_mtip* h);
int spf_mtip_set_orientations(spf_mtip* h, const float* quats, const float* q_lab, void* stream);
int spf_mtip_set_mask(spf_mtip* h, const float* D, void* stream);
int spf_mtip_match(spf_mtip* h, const float* A, const void* images, int image_type, int n_img, float img_scale,
                   int32_t* best, float* best_d, float* second_d, int32_t* topk_idx, float* topk_d, void* stream);
int spf_mtip_merge(spf_mtip* h, const void* images, int image_type, int n_img, float img_scale, const int32_t* best,
                   float* rhs, float* kernel_hat, void* stream);
int spf_mtip_solve(spf_mtip* h, const float* rhs, const float* kernel_hat, const float* x0, double lam_rel,
                   int64_t n_img_total, int cg_iters, float* x, double* lambda_out, double* res_hist, void* stream);
int spf_mtip_iteration(spf_mtip* h, const float* A, const void* images, int image_type, int n_img, float img_scale,
                       int cg_iters, double lam_rel, int32_t* best, float* x, double* lambda_out, void* stream);
int spf_mtip_iteration_host(spf_mtip* h, const float* A_host, const void* images_host, int image_type, int n_img,
                            float img_scale, int cg_iters, double lam_rel, int32_t* best_host, float* x_host,
                            double* lambda_out, void* stream);
int spf_mtip_set_upload(spf_mtip* h, int mode);
int spf_mtip_last_upload_ms(spf_mtip* h, float* ms);
int spf_mtip_upload_host(spf_mtip* h, const float* A_host, const void* images_host, int image_type, int n_img,
                         float** A_dev, const void** images_dev, void* stream);
int spf_mtip_release_upload(spf_mtip* h, void* stream);

/* ---------------------------------------------------------------------------
 * Phasing, Sec. II-D: from the merged diffraction volume to a density by
 * error reduction (ER), hybrid input-output (HIO) and shrinkwrap, the
 * published methods the paper combines, on the model's N^3 grid (N odd,
 * 3..401; layout as the model). Transforms are exact DFTs:
 *   forward rho^_m = sum_n rho_n exp(-2 pi i m.n / N),
 *   inverse rho_n  = N^-3 sum_m rho^_m exp(+2 pi i m.n / N).
 * Data: magnitudes amp_m (amp < 0: a mode without data, left free).
 *   P_M rho: rho^ -> amp rho^ / |rho^| on modes with data (amp where
 *            rho^ = 0), back to real space (real part).
 *   ER:  rho' = P_M rho where (support and, with positivity, P_M rho > 0),
 *        else 0.
 *   HIO: the same where kept, else rho - beta P_M rho.
 *   Fourier error of an iterate: sqrt(sum_data (|rho^| - amp)^2 / sum_data amp^2).
 *   Shrinkwrap: support = blur > threshold * max(blur), blur = |rho|
 *        circularly convolved with the normalised Gaussian of width sigma
 *        voxels over the minimal periodic offsets {-M..M}^3.
 * spf_phaser_create allocates the iterate, support (initially all ones),
 *   magnitudes, work cube and scratch (about 30 bytes per voxel).
 * spf_phaser_set_amplitudes copies amp (N^3 floats, device);
 * spf_phaser_amplitudes_from_model sets amp = sqrt(max(Re forward(x), 0))
 *   from a merged autocorrelation x (N^3 floats, device): every mode has data.
 * spf_phaser_set_state copies the iterate rho (N^3 floats) and / or the
 *   support (N^3 bytes, nonzero = inside); either may be NULL.
 * spf_phaser_iterate: `iters` steps of SPF_PHASE_ER or SPF_PHASE_HIO (beta
 *   used by HIO), positivity 0 / 1; errors (device, iters doubles, may be
 *   NULL) receives the Fourier error of each iterate before its step.
 * spf_phaser_shrinkwrap updates the support from the current iterate.
 * spf_phaser_get copies the iterate, support and magnitudes out (each
 *   device pointer may be NULL).
 * All stream-ordered; FP32 transforms, FP64 error sums.
 * ------------------------------------------------------------------------- */
#define SPF_PHASE_ER 0
#define SPF_PHASE_HIO 1
typedef struct spf_phaser spf_phaser;
int spf_phaser_create(spf_phaser** out, int N, int device);
int spf_phaser_destroy(spf_phaser* ph);
int spf_phaser_set_amplitudes(spf_phaser* ph, const float* amp, void* stream);
int spf_phaser_amplitudes_from_model(spf_phaser* ph, const float* x, void* stream);
int spf_phaser_set_state(spf_phaser* ph, const float* rho, const uint8_t* support, void* stream);
int spf_phaser_iterate(spf_phaser* ph, int method, int iters, float beta, int positivity, double* errors,
                       void* stream);
int spf_phaser_shrinkwrap(spf_phaser* ph, float sigma, float threshold, void* stream);
int spf_phaser_get(spf_phaser* ph, float* rho, uint8_t* support, float* amp, void* stream);

/* ---------------------------------------------------------------------------
 * Photon-count images (no counterpart in the paper's equations; its images
 * are photon counts). Moving frames as 16-bit counts halves the
 * host-to-device bytes of FP32 images; the FP32 copy the other calls take is
 * made on the device.
 * spf_counts_to_f32: out[i] = (float)counts[i] for 0 <= i < n. counts: n
 *   unsigned 16-bit values, 2-byte aligned; out: n floats; both device
 *   pointers, not overlapping, caller-owned. Asynchronous on `stream`.
 *   SPF_ERR_ARG for n < 0 or a NULL pointer with n > 0.
 * ------------------------------------------------------------------------- */
int spf_counts_to_f32(const uint16_t* counts, int64_t n, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Matching without device allocation. The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc when they match -- code inside a
 * host framework that owns the device memory pool and forbids allocations
 * beside it (its allocator must account for every byte), or a real-time
 * acquisition loop that must not touch the allocator, whose calls can block
 * and synchronise the device. It computes what spf_match_orientations
 * computes with precision SPF_FP32 and topk 8 (fused FP32 distance + top-8,
 * exact FP32 re-rank), but every intermediate buffer lives in one static
 * device array of 4,526,080 bytes (about 4.5 MB) that each GPU loading this
 * library holds until the process exits.
 *   images: n_img x P2, slices: n_orient x P2, outputs: n_img each (device).
 *   n_img <= SPF_STATIC_MATCH_MAX_IMAGES, n_orient <= SPF_STATIC_MATCH_MAX_ORIENT;
 *   larger sizes return SPF_ERR_ARG with a message.
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); it is looked up again when the
 * calling thread's current CUDA context changes (for instance after
 * cudaDeviceReset). Make that first call before any stream capture. It
 * allocates nothing, then or later. Every call resets the part of the array
 * it reads before use. All calls on a device share the one array: calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and give wrong results -- serialise them. Runs on the calling thread's
 * current device.
 * ------------------------------------------------------------------------- */
#define SPF_STATIC_MATCH_MAX_IMAGES 1024
#define SPF_STATIC_MATCH_MAX_ORIENT 65536
int spf_match_orientations_static(const float* images, int n_img, float img_scale,
                                  const float* slices, int n_orient, int P2, int32_t* best_idx,
                                  float* best_d, float* second_d, void* stream);

/* ---------------------------------------------------------------------------
 * Tracing (no counterpart in the paper; it backs the per-stage timings of
 * its Fig. 5 style breakdown). Host calls.
 * spf_profile_enable(1) clears the counters and starts recording a CUDA event
 *   pair around every kernel launch on the launching stream; 0 stops.
 * spf_profile_read: for kernel number `index` (0 ..), its name (copied into
 *   name[0..name_len-1]), launches and summed device milliseconds since the
 *   last enable. Waits for the recorded events. SPF_ERR_ARG past the last.
 * spf_profile_select: restrict the event pairs to the kernels named in the
 *   comma-separated list `names` (NULL or "" selects every kernel); the
 *   other launches are still counted by spf_launch_count. Lets a caller time
 *   one kernel inside a timed region without an event pair on every launch.
 * spf_profile_bytes: for kernel number `index`, the algorithmic global-memory
 *   bytes of its traced launches since the last enable (each input element
 *   read once and each output element written once, as the launch site
 *   states it; 0 for kernels that state none). The bandwidth-bound kernels
 *   (FFT passes, padding and cropping, CG vectors) state theirs.
 * spf_launch_count: kernels launched by this library since the process began.
 * ------------------------------------------------------------------------- */
int spf_profile_enable(int on);
int spf_profile_select(const char* names);
int spf_profile_read(int index, char* name, int name_len, long long* launches, double* total_ms);
int spf_profile_bytes(int index, double* bytes);
long long spf_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SPF_H */
