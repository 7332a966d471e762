/*
 * shine.h -- C ABI of the fused Harris pattern pipeline on one GPU (sm_103a).
 *
 * The pipeline is a composition of data-parallel patterns applied to an RGB image:
 *
 *   A1  G  = map(grayscale)(img)                       gray = 0.299 r + 0.587 g + 0.114 b
 *   A2  Ix = map(reduce(+) . zip(W_x))(slide2D(3,1)(pad(G)))      and Iy with W_y
 *   A3  P  = map((ix, iy) -> (ix*ix, ix*iy, iy*iy))(zip(Ix, Iy))
 *   A4  S  = map(reduce(+))(slide2D(3,1)(pad(P)))       unnormalised 3x3 box sum, per plane
 *   A5  R  = map((sxx, sxy, syy) -> sxx*syy - sxy^2 - kappa*(sxx+syy)^2)(S)
 *
 * map, zip and reduce are the RISE primitives of the paper (Sec. 4.1); fusing the stages
 * into one kernel with no intermediate buffer follows its map-fusion and fuseReduceMap
 * rewrite rules (Sec. 4.2); only the result is written to global memory (toMem(Global),
 * Sec. 5.3). slide2D(3,1) makes the 3x3 windows window[a][b] = x[i+a][j+b]; the weights are
 * applied as a correlation (window[a][b] * W[a][b]); x is the column index.
 *
 * Borders.  SHINE_VALID: no padding; each 3x3 stage shrinks by 2, the output is (H-4) x (W-4)
 * and needs H, W >= 5.  SHINE_CLAMP: pad_clamp2D(1) before each 3x3 stage (index clamp(i-1,
 * 0, n-1)), so the output is H x W for any H, W >= 1. The products are clamped at their own
 * stage, not recomputed from a further-clamped gray image.
 *
 * Layouts.  Images are H rows of W pixels, each pixel 3 interleaved channels (r, g, b),
 * row-major, channel fastest; img_pitch is the distance between rows in ELEMENTS (>= 3W).
 * Outputs and cotangents are H_out x W_out single-channel maps with their own pitch in
 * elements (>= W_out). Weights wx, wy are 3x3 row-major float32 (wx[3a + b] = W_x[a][b]);
 * kappa is one float32. All pointers are DEVICE pointers unless marked (host); every buffer
 * is owned by the caller. Arithmetic is float32 whatever the storage type; the response
 * step A5 is always float32.
 *
 * Fast-path alignment.  Rows are staged with 16-byte (float32) or 8-byte (bf16/fp16) copies
 * when the image pointer and img_pitch * sizeof(element) are multiples of that size, and
 * stored with 16- / 8-byte stores when the output pointer and pitch allow; otherwise the call
 * takes an element-wise path that gives identical results, more slowly.
 *
 * Errors.  Argument errors are detected on the host and returned before anything is
 * launched; launch failures come back as SHINE_ERR_CUDA (the CUDA error is then available
 * from shine_last_cuda_error). Fault injection for callers' error paths: with the environment
 * variable SHINE_FAULT_INJECT="<call>=<status>[,...]" ("*" names every call), each named compute
 * entry point returns that status (1..5) at once, before reading its arguments or touching the
 * GPU. Each compute entry point also opens an NVTX range named after itself (free unless a
 * profiler is attached). Calls are asynchronous on the given stream, never
 * synchronise, never allocate (except shine_plan_create), never throw, and are reentrant.
 * Gradients are OVERWRITTEN, not accumulated; a NULL gradient pointer skips that output.
 */
#ifndef SHINE_H_
#define SHINE_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SHINE_API __attribute__((visibility("default")))
#else
#define SHINE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SHINE_OK = 0,
    SHINE_ERR_INVALID_ARG = 1,  /* NULL pointer, bad enum, bad shape or pitch */
    SHINE_ERR_ALIGNMENT = 2,    /* a pointer that must be 4-byte aligned is not */
    SHINE_ERR_WORKSPACE = 3,    /* workspace missing or smaller than required */
    SHINE_ERR_UNSUPPORTED = 4,  /* a combination this build does not implement */
    SHINE_ERR_CUDA = 5          /* a CUDA call or kernel launch failed */
} shine_status;

typedef enum { SHINE_F32 = 0, SHINE_BF16 = 1, SHINE_F16 = 2 } shine_dtype;
typedef enum { SHINE_VALID = 0, SHINE_CLAMP = 1 } shine_border;

/* Output size of the pipeline for an H x W image (host helper; 0 on success). */
SHINE_API shine_status shine_output_shape(int64_t H, int64_t W, shine_border border, int64_t* H_out,
                                int64_t* W_out);

/*
 * Forward pass: R = A5(A4(A3(A2(A1(img))))) in one fused kernel (no intermediate in HBM).
 *   img       [H][img_pitch] elements of type dt (3 channels per pixel)
 *   kappa     [1] float32, wx/wy [9] float32 (device)
 *   out       [H_out][out_pitch] elements of type out_dt
 *   stream    a cudaStream_t (NULL = legacy default stream)
 * Shapes: H, W >= 1 (CLAMP) or >= 5 (VALID); H, W <= 2^30; pitches >= 3W and >= W_out.
 */
SHINE_API shine_status shine_pipeline_fwd(const void* img, int64_t H, int64_t W, int64_t img_pitch,
                                shine_dtype dt, shine_border border, const float* kappa,
                                const float* wx, const float* wy, void* out, int64_t out_pitch,
                                shine_dtype out_dt, void* stream);

/*
 * Forward and backward in one pass, for when the cotangent grad_out is known before R is
 * needed (a loss sum(w * R) with fixed weights w): writes R (type dt, nullable) and the same
 * cotangents as shine_pipeline_bwd. Reads the image and grad_out once and writes R and
 * grad_img once; uses the workspace size of shine_pipeline_bwd_workspace.
 */
SHINE_API shine_status shine_pipeline_fwd_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch,
                                    shine_dtype dt, shine_border border, const float* kappa,
                                    const float* wx, const float* wy, const void* grad_out,
                                    int64_t gout_pitch, void* out, int64_t out_pitch,
                                    void* grad_img, int64_t gimg_pitch, float* grad_kappa,
                                    float* grad_wx, float* grad_wy, void* workspace,
                                    size_t ws_bytes, void* stream);

/* Workspace (bytes, host out-param) that shine_pipeline_bwd needs for an H x W image. */
SHINE_API shine_status shine_pipeline_bwd_workspace(int64_t H, int64_t W, shine_border border,
                                          size_t* bytes);

/*
 * Backward pass (vector-Jacobian product) of L = sum(grad_out * R): reverse mode through the
 * same patterns -- each stencil's adjoint is its transposed stencil (overlap-add), each clamp
 * pad's adjoint folds the padded cotangent onto the clamped index, and the shared parameters'
 * cotangents are sums over all pixels. The Sobel stage is recomputed, not read back.
 *   grad_out   [H_out][gout_pitch] of type gout_dt (device)
 *   grad_img   [H][gimg_pitch] of type dt, 3 channels per pixel (nullable)
 *   grad_kappa [1], grad_wx [9], grad_wy [9] float32 (each nullable)
 *   workspace  at least shine_pipeline_bwd_workspace() bytes of device memory, 16-byte
 *              aligned; its contents are scratch (per-tile partial sums)
 * The parameter cotangents are reduced in a fixed order in float64, so repeated calls give
 * bit-identical results. Kernel choice: 16-bit CLAMP images whose image and cotangent rows are
 * 16-byte aligned take the eight-columns-per-lane kernel from 2^25 pixels on (the environment
 * variable SHINE_WIDE_BWD_MIN_PIXELS, read at every call, moves that bound); R and d img are
 * bit-identical either way, the parameter cotangents are the same terms summed over another
 * partition. The same holds for shine_pipeline_fwd_bwd.
 */
SHINE_API shine_status shine_pipeline_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch,
                                shine_dtype dt, shine_border border, const float* kappa,
                                const float* wx, const float* wy, const void* grad_out,
                                int64_t gout_pitch, shine_dtype gout_dt, void* grad_img,
                                int64_t gimg_pitch, float* grad_kappa, float* grad_wx,
                                float* grad_wy, void* workspace, size_t ws_bytes, void* stream);

/*
 * Forward and backward of an image held in HOST memory: uploads, kernels and downloads are cut
 * into nbands row bands and overlapped on the library's own streams (band b's kernels run once
 * band b+1, holding its halo rows, has arrived), so the call costs about one transfer direction
 * instead of the sum of both. Results equal those of shine_pipeline_fwd + shine_pipeline_bwd.
 *   img_h, gout_h          host inputs, dense rows (pitch 3W / W_out elements); pinned memory
 *                          is needed for the copies to overlap
 *   out_h, gimg_h          host outputs (dense; each nullable)
 *   kappa, wx, wy          device parameters
 *   grad_params            device float32 [19]: d kappa, d Wx[9], d Wy[9] (nullable)
 *   dev_img, dev_gout, dev_out, dev_gimg
 *                          device buffers of the full sizes (dense, 16-byte aligned)
 *   workspace              >= shine_pipeline_host_workspace() bytes of device memory
 *   nbands                 1..64, and H >= 8 * nbands
 * The caller's stream waits for all of it (copies included): synchronise that stream before
 * reading the host outputs. One call at a time per device.
 */
SHINE_API shine_status shine_pipeline_host_workspace(int64_t H, int64_t W, shine_border border,
                                          int32_t nbands, size_t* bytes);
SHINE_API shine_status shine_pipeline_host(const void* img_h, const void* gout_h, void* out_h,
                                 void* gimg_h, int64_t H, int64_t W, shine_dtype dt,
                                 shine_border border, const float* kappa, const float* wx,
                                 const float* wy, float* grad_params, void* dev_img,
                                 void* dev_gout, void* dev_out, void* dev_gimg, void* workspace,
                                 size_t ws_bytes, int32_t nbands, void* stream);

/*
 * Backward pass that allocates nothing, for callers that cannot allocate device memory (a
 * plug-in handed only its input and output buffers, a real-time loop that forbids allocation
 * after start-up, code inside a framework that owns all device memory). The paper has no
 * counterpart; this is an interface convenience of this library.
 *
 * Same arguments and results as shine_pipeline_bwd, without the workspace: the per-warp partial
 * sums live in one fixed array of the library's device memory (about 2.5 MB: 19 x 16384
 * doubles), held on every GPU that loads the library until the process exits. Returns
 * SHINE_ERR_UNSUPPORTED when an image would need more partial sums than that array holds (not
 * reached on GPUs with up to 256 SMs). The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first call before any stream
 * capture. All calls share the one array: calls whose GPU work can overlap in time (different
 * streams without ordering between them, or several host threads) race on it and give wrong
 * cotangents; serialise them on one stream. Nothing needs clearing between calls. A bounded
 * wait that gives up (results invalid) is reported through shine_wait_status, like the calls
 * without a workspace, not through shine_workspace_status.
 */
SHINE_API shine_status shine_pipeline_bwd_noalloc(const void* img, int64_t H, int64_t W, int64_t img_pitch,
                                    shine_dtype dt, shine_border border, const float* kappa,
                                    const float* wx, const float* wy, const void* grad_out,
                                    int64_t gout_pitch, shine_dtype gout_dt, void* grad_img,
                                    int64_t gimg_pitch, float* grad_kappa, float* grad_wx,
                                    float* grad_wy, void* stream);

/*
 * Many images of different sizes in one persistent launch.
 *
 * shine_plan_create builds, on the host and then once on the device, the tile list of a fixed
 * set of image shapes (HW: host array of n (H, W) pairs), choosing the tile height per shape
 * bucket and the schedule (see shine_plan_schedule) from tune_cache_path when given and it holds
 * entries for this GPU, else built-in rules. Cache lines (text, '#' comments):
 *   <gpu key> <dtype> <border> <mode> <bucket> <band_rows>      bucket = ceil(log2(rows))
 *   <gpu key> <dtype> <border> <mode> plan <order> <staging> <edge_w4> <origin> mode: SHINE_MODE_FWD computes R only; SHINE_MODE_FWD_BWD also computes the
 * cotangents of L = sum_i sum(grad_out_i * R_i) in the same pass (grad_out is an input given
 * up front). This is the only call that allocates (host memory and one device buffer).
 */
typedef struct shine_plan shine_plan;
enum { SHINE_MODE_FWD = 1, SHINE_MODE_FWD_BWD = 3 };

typedef struct {
    const void* img;       /* [H][img_pitch], 3 channels, plan dtype */
    void* out;             /* [H_out][out_pitch], plan dtype (nullable in FWD_BWD mode) */
    const void* grad_out;  /* [H_out][gout_pitch], plan dtype (FWD_BWD mode) */
    void* grad_img;        /* [H][gimg_pitch], plan dtype (FWD_BWD mode, nullable) */
    int64_t H, W;
    int64_t img_pitch, out_pitch, gout_pitch, gimg_pitch;
} shine_image_desc;

SHINE_API shine_status shine_plan_create(const int64_t* HW, int32_t n, shine_dtype dt, shine_border border,
                               int32_t mode, const char* tune_cache_path, shine_plan** plan);

/* Device workspace (bytes) the batched call needs for this plan. */
SHINE_API shine_status shine_plan_workspace(const shine_plan* plan, size_t* bytes);

/* Tile height the plan chose for image i (host; for tests and reports). */
SHINE_API shine_status shine_plan_tile_rows(const shine_plan* plan, int32_t i, int32_t* rows);

/*
 * The schedule the plan chose (host; no counterpart in the paper): the order in which the
 * persistent warps claim the tiles (SHINE_ORDER_*: longest tile first, image by image, or the
 * images with the most work first), the staging of interior segments in SHINE_MODE_FWD_BWD
 * (0: every lane copies its own chunks with cp.async; 1: bulk copies by one lane, for images
 * whose image and cotangent rows are 16-byte aligned), the weight of an edge-segment tile row
 * against an interior one (edge_w4 / 4) in the claim order's work estimate, and the first output
 * column of segment 0 of every image (segments are 120 columns wide). All four come from the
 * tuning cache's "plan" line when it has one for this GPU, else from the defaults (longest
 * first, cp.async, 6, 0).
 */
enum { SHINE_ORDER_LONGEST_FIRST = 0, SHINE_ORDER_IMAGE = 1, SHINE_ORDER_LARGEST_IMAGE_FIRST = 2 };
SHINE_API shine_status shine_plan_schedule(const shine_plan* plan, int32_t* order, int32_t* staging,
                                           int32_t* edge_w4, int32_t* origin);

/*
 * Run the plan: descs is a DEVICE array of n image descriptors (same order and shapes as at
 * plan creation), kappa [n] one per image, wx/wy [9] shared by every image. grad_kappa [n],
 * grad_wx [9], grad_wy [9] are float32 outputs (nullable; FWD_BWD mode). Launches a
 * persistent kernel (one CTA per SM slot, tiles claimed from an atomic counter in the
 * workspace) and a fixed-order reduction; no allocation and no synchronisation, so the call
 * can be captured in a CUDA graph. Results do not depend on which CTA ran which tile. A bounded
 * wait of bulk staging that gives up (results invalid) sets the workspace's first word, which
 * shine_workspace_status reads.
 */
SHINE_API shine_status shine_pipeline_batched(const shine_plan* plan, const shine_image_desc* descs,
                                    const float* kappa, const float* wx, const float* wy,
                                    float* grad_kappa, float* grad_wx, float* grad_wy,
                                    void* workspace, size_t ws_bytes, void* stream);

SHINE_API void shine_plan_destroy(shine_plan* plan);

/*
 * Key under which the tuning cache stores entries for the current device (host call): GPU
 * name, compute capability, SM count and CUDA runtime version. Writes at most len bytes
 * (NUL-terminated) to buf and returns the key's length, or -1 when no device is visible.
 */
SHINE_API int shine_tune_key(char* buf, size_t len);

/*
 * Corner detection: the forward pass followed, in the same kernel, by a threshold and a 3x3
 * non-maximum suppression of R (one more map over slide2D(3,1) windows, fused after A5):
 *   mask[y][x] = 1  if R[y][x] > threshold and R[y][x] >= R at each of its 8 neighbours that
 *                   lie inside the output region (neighbours outside it are ignored),
 *                0  otherwise.
 * R is the value shine_pipeline_fwd computes, bit for bit (same kernel arithmetic); ties keep
 * every tied maximum. A NaN R is never a corner.
 *   mask       [H_out][mask_pitch] bytes (uint8, device), mask_pitch >= W_out
 *   out        optional R, as in shine_pipeline_fwd (NULL: R is not written; out_dt ignored)
 *   threshold  host float32 value
 * Other arguments, shapes and errors as in shine_pipeline_fwd; mask must not be NULL.
 */
SHINE_API shine_status shine_corners(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                     shine_border border, const float* kappa, const float* wx, const float* wy,
                                     float threshold, uint8_t* mask, int64_t mask_pitch, void* out,
                                     int64_t out_pitch, shine_dtype out_dt, void* stream);

/*
 * Harris with a weighted window: the forward pipeline with its A4 box replaced by a separable
 * K-tap window (K = 3, 5, 7; e.g. Gaussian taps), fused into one kernel like the forward:
 *   A1 gray, A2 3x3 Sobel (Wx, Wy, per-stage clamp), A3 products,
 *   A4' S_c = sum_{a,b} gv[a] gh[b] P_c[clamp(i-r+a)][clamp(j-r+b)]   (r = (K-1)/2; computed as
 *       the column sum with gv, then the row sum with gh, each a float32 fma chain from zero),
 *   A5 R = Sxx Syy - Sxy^2 - kappa (Sxx + Syy)^2.
 * CLAMP borders only (output H x W). gv, gh: HOST pointers to K float32 each (copied at the
 * call). dt/out_dt: F32 -> F32, BF16 -> BF16 or F32. Other arguments as shine_pipeline_fwd.
 * Errors: K not in {3, 5, 7}, bad shapes or NULL pointers -> SHINE_ERR_INVALID_ARG; other dtype
 * pairs -> SHINE_ERR_UNSUPPORTED; misaligned pointers -> SHINE_ERR_ALIGNMENT.
 */
SHINE_API shine_status shine_harris_window(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                           const float* kappa, const float* wx, const float* wy, int32_t K,
                                           const float* gv, const float* gh, void* out, int64_t out_pitch,
                                           shine_dtype out_dt, void* stream);

/*
 * Generalised stencil: one fused slide2D(K, 1) + reduce stage over a single-channel array,
 *   out = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(K, 1)(pad(in)))
 * K odd, 1 <= K <= 9, r = (K-1)/2; SHINE_CLAMP pads with pad_clamp2D(r) (output H x W),
 * SHINE_VALID does not pad (output (H-2r) x (W-2r), needs H, W >= K). The weights act as a
 * correlation: out[i][j] = sum_{a,b} W[a][b] * in_padded[i+a][j+b].
 *   weights  HOST pointer to K*K float32, row-major (W[a][b] = weights[a*K + b]); or NULL for
 *            the separable form, which then takes
 *   wv, wh   HOST pointers to K float32 each: a K-tap stage down the columns with wv, then a
 *            K-tap stage along the rows with wh (the composition of two 1-D slide + reduce
 *            stages; equal to W = wv wh^T up to rounding).
 * The weights are copied at the call into the kernel's parameters (they are not read later).
 *   in   [H][in_pitch] elements of dt (device), out [H_out][out_pitch] of out_dt (device)
 *   dt/out_dt: F32 -> F32, BF16 -> BF16 or F32 (float32 arithmetic throughout).
 * Each output is a float32 fused multiply-add chain over its taps in row-major order from zero
 * (separable: the column chain, then the row chain). Errors: bad K, shapes, pitches or NULL
 * pointers -> SHINE_ERR_INVALID_ARG; other dtype pairs -> SHINE_ERR_UNSUPPORTED; misaligned
 * elements -> SHINE_ERR_ALIGNMENT.
 */
SHINE_API shine_status shine_stencil2d(const void* in, int64_t H, int64_t W, int64_t in_pitch, shine_dtype dt,
                                       shine_border border, int32_t K, const float* weights, const float* wv,
                                       const float* wh, void* out, int64_t out_pitch, shine_dtype out_dt,
                                       void* stream);

/*
 * iterate with double buffering (Sec. 6): k rounds of the body split(n) >> map(reduce(+, 0))
 * applied to Array[(n^k) * m], so that
 *   out[j] = the level-by-level tree sum of in[j * n^k .. (j+1) * n^k): every round replaces
 *            each n consecutive values by their left fold from 0 (((0 + a0) + a1) + ...).
 *   in   [(n^k) * m] float32 (device), out [m] float32 (device, overwritten)
 * The rounds ping-pong between two shared-memory buffers: round 0 reads the input straight
 * from global memory, the last round writes out; every sum keeps the fold order above, so the
 * result equals a float32 evaluation of the definition bit for bit. k == 0 copies m values.
 * Limits: n >= 1, k >= 0, (n^k) * m <= 2^40; one group's n^(k-1) round-1 values must fit one
 * buffer (6144 floats) when k > 1, else SHINE_ERR_UNSUPPORTED. Errors: bad sizes or NULL
 * pointers -> SHINE_ERR_INVALID_ARG; in/out not 4-byte aligned -> SHINE_ERR_ALIGNMENT.
 */
SHINE_API shine_status shine_iterate_sum(const float* in, int64_t m, int32_t n, int32_t k, float* out, void* stream);

/*
 * The same iterate with the body split(n) >> map(reduce(op, identity)): op SHINE_REDUCE_SUM
 * (+ from 0; shine_iterate_sum), SHINE_REDUCE_MAX (max from -inf) or SHINE_REDUCE_MIN (min from
 * +inf). max and min are IEEE maxNum / minNum (a NaN operand is ignored unless both are NaN) and
 * exact, so their results do not depend on the grouping. Arguments, limits and errors as
 * shine_iterate_sum; an unknown op -> SHINE_ERR_INVALID_ARG.
 */
typedef enum { SHINE_REDUCE_SUM = 0, SHINE_REDUCE_MAX = 1, SHINE_REDUCE_MIN = 2 } shine_reduce_op;
SHINE_API shine_status shine_iterate_reduce(const float* in, int64_t m, int32_t n, int32_t k, shine_reduce_op op,
                                            float* out, void* stream);

/*
 * iterate with a size-preserving body (Sec. 6, n = 1): k rounds of the clamp-padded 3x3 stencil
 *   x_{i+1} = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))
 *             (slide2D(3, 1)(pad_clamp2D(1)(x_i))),   x_0 = in,  out = x_k
 * (an iterated blur when the weights are a smoothing kernel). Clamp padding applies before every
 * round; W acts as a correlation, W[a][b] on x_i[y + a - 1][x + b - 1] (clamped).
 *   in  [H][in_pitch] float32 (device; row y at in + y * in_pitch), read only
 *   out [H][out_pitch] float32 (device, overwritten; must not overlap in)
 *   weights [9] float32, HOST memory, row-major, copied at the call
 * The double buffer lives in shared memory per 64 x 112 output tile (temporal blocking): round 0
 * reads in straight from global memory, the rounds between ping-pong in shared memory, round k-1
 * writes out. Each output is a chain of float32 fused multiply-adds per round (taps in row-major
 * order from zero). Limits: 1 <= k <= 8; 1 <= H, W <= 2^30; pitches >= W. Errors: NULL pointers,
 * bad sizes or overlapping in/out -> SHINE_ERR_INVALID_ARG; in/out not 4-byte aligned ->
 * SHINE_ERR_ALIGNMENT. Asynchronous on `stream`; no allocation.
 */
SHINE_API shine_status shine_iterate_stencil(const float* in, int64_t H, int64_t W, int64_t in_pitch,
                                             const float* weights, int32_t k, float* out, int64_t out_pitch,
                                             void* stream);

/*
 * Matrix-vector multiply, the paper's running example (Sec. 4, MV):
 *   y[i] = reduce(+, 0)(map(*)(zip(A[i], x)))  =  sum_j A[i][j] * x[j]
 *   A      [M][lda] elements of type dt, row-major, lda >= max(N, 1) (device)
 *   x      [N] float32 (device), y [M] float32 (device, overwritten; N == 0 gives zeros)
 *   stream a cudaStream_t
 * A row's reduce is split across the 32 lanes of a warp: lane l sums, with float32 fused
 * multiply-adds in order, the 16-byte chunks l, l+32, ... of the row into four accumulators
 * (chunk c into accumulator (c / 32) mod 4; elements past the last whole chunk by the lane
 * that owns them), adds them as (a0 + a1) + (a2 + a3), and the 32 lane sums are combined by a
 * fixed butterfly; results do not depend on the launch and repeat bit for bit. Rows are read
 * once from HBM (16-byte streaming loads when A, lda * sizeof(dt) and x allow; element loads
 * otherwise, summed per lane in element order). Shapes: 0 <= M, N <= 2^31. Errors: invalid
 * shapes or NULL pointers -> SHINE_ERR_INVALID_ARG; A not aligned to its element size or x,
 * y not 4-byte aligned -> SHINE_ERR_ALIGNMENT.
 */
SHINE_API shine_status shine_mv(const void* A, int64_t M, int64_t N, int64_t lda, shine_dtype dt, const float* x,
                                float* y, void* stream);

/*
 * Bounded waits. Every wait of the kernels on a bulk copy polls its barrier a bounded number of
 * times; a wait that gives up stops its warp's work (the results of that call are invalid) and
 * sets a flag instead of hanging the GPU. Calls with a workspace (the backward passes) report it
 * through shine_workspace_status; the forward, corner and window calls and
 * shine_pipeline_bwd_noalloc set one library-wide flag per GPU, read (and cleared when
 * clear != 0) by shine_wait_status. Both synchronise with the device.
 */
SHINE_API shine_status shine_wait_status(int* failed, int clear);

/*
 * Index checks of debug builds (no counterpart in the paper; a stand-in for a memory checker).
 * The library built with SHINE_DEBUG_BOUNDS=1 (libshine_debug.so) checks the row and column
 * ranges of the Harris kernels' global loads, stores and copies and of their shared-memory
 * staging, and on a violation sets a bit of one word per GPU (bit 0 forward loads, 1 forward
 * stores, 2 forward copies, 3 adjoint copies, 4 adjoint stores, 5 shared memory) without
 * trapping. *instrumented is 1 in such a build, 0 otherwise (then *bits is always 0); *bits is
 * the word, cleared when clear != 0. Synchronises with the device in a debug build.
 */
SHINE_API shine_status shine_debug_bounds_status(int* instrumented, unsigned int* bits, int clear);

/*
 * Host-side view of the work partition the kernels use (no counterpart in the paper; for tests
 * and tuning): the (segment, row) units [*lo, *hi), in segment-major order, that warp w of t
 * takes over nseg column segments of rows rows; band_major != 0 selects the band-major layout
 * (one segment and one row band per warp when t >= nseg), edge_weight4 / 4 is the weight of an
 * edge-segment row against an interior row (4: unweighted). No GPU is touched.
 */
SHINE_API shine_status shine_partition(int64_t nseg, int64_t rows, int64_t t, int64_t w, int32_t band_major,
                                       int32_t edge_weight4, int64_t* lo, int64_t* hi);

/*
 * Self-test of the bounded-wait path (no counterpart in the paper): launches one warp that
 * waits, with at most max_spins polls (1 .. 2^22), on a shared-memory barrier that nothing
 * completes, and writes 1 to *result (a device int) when the wait gave up -- as it must -- and
 * 0 otherwise. No fault is involved; the context stays usable. Asynchronous on stream.
 */
SHINE_API shine_status shine_selftest_bounded_wait(int32_t max_spins, int* result, void* stream);

/* Static description of a status code. */
SHINE_API const char* shine_status_string(shine_status s);

/* The cudaError_t (as int) of the last SHINE_ERR_CUDA returned on this host thread. */
SHINE_API int shine_last_cuda_error(void);

/*
 * Whether the last backward pass run on this workspace gave up waiting for its staged rows
 * (*failed = 1; its results are then not valid) -- every wait in the kernels is bounded, so a
 * fault of the copy engine surfaces here instead of as a hang. Synchronises with the device.
 */
SHINE_API shine_status shine_workspace_status(const void* workspace, int* failed);

#ifdef __cplusplus
}
#endif

#endif /* SHINE_H_ */
