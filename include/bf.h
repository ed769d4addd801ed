/*
 * bf.h -- C ABI of libbf, a GB300 (sm_103a) implementation of the Monte Carlo
 * shiftable bilateral filter for vector-valued images (Ghosh & Chaudhury,
 * "Fast Bilateral Filtering of Vector-Valued Images", arXiv 1605.02164).
 *
 * The filter (Eqs. BF, normal) is
 *     B[f](i) = sum_j w(j) phi(f(i-j) - f(i)) f(i-j) / sum_j w(j) phi(f(i-j) - f(i)),
 *     w(j) = exp(-|j|^2 / (2 sigma_s^2)),  phi(x) = exp(-x^T C^{-1} x / 2),
 * over the window |j_x|, |j_y| <= r = floor(3 sigma_s) (Section 1), leaving out
 * neighbours outside the image.  libbf computes the paper's approximation
 * (Algorithm 1, Eqs. numerator and denom): the range kernel is whitened, each
 * 1-D Gaussian is replaced by a raised cosine of order N (Eq. approx), and the
 * product of raised cosines is sampled with K = T Monte Carlo draws
 * (Prop. 2, Eq. finalApproxY).  With nu_t = W^T Y_t / (2 pi sqrt(N)) the output is
 *     S_c(i) = Re P_c(i) / Re Z(i),
 *     P_c(i) = sum_t sum_j w(j) cos(2 pi nu_t . (f(i-j) - f(i))) f_c(i-j),
 *     Z(i)   = sum_t sum_j w(j) cos(2 pi nu_t . (f(i-j) - f(i))),
 * evaluated in shiftable form: per term, 2(d+1) modulated channels
 * (cos th f_c, sin th f_c, cos th, sin th) are blurred by the Gaussian and
 * combined with the centre pixel's cos th and sin th.
 *
 * Conventions for every call:
 *   - Return value: BF_OK (0) on success, else one negative BF_ERR_* code.
 *     Nothing is written to outputs on a host-side error.
 *   - Images are FP32, planar [d][H][pitch] (element (c, y, x) at
 *     base[c*H*pitch + y*pitch + x]), on the device unless the call says host.
 *     The caller owns image buffers and streams; libbf owns plans and its
 *     internal scratch.
 *   - Filtering calls are asynchronous on the given stream (NULL = legacy
 *     default stream) and launch only CUDA kernels of this library; there is
 *     no CPU fallback.  Input and output must not overlap (no in-place).
 *   - A stream argument is a cudaStream_t passed as void*.
 */
#ifndef BF_H_
#define BF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define BF_OK 0
#define BF_ERR_ARG (-1)         /* null pointer, bad size, overlap, bad enum */
#define BF_ERR_NOT_SPD (-2)     /* C is not symmetric positive definite */
#define BF_ERR_D_RANGE (-3)     /* d outside [1, BF_MAX_D] */
#define BF_ERR_ALIGN (-4)       /* pointer or pitch misaligned */
#define BF_ERR_NOMEM (-5)       /* device or host allocation failed */
#define BF_ERR_BUDGET (-6)      /* request exceeds a memory budget */
#define BF_ERR_TIMEOUT (-7)     /* a bounded device-side wait ran out */
#define BF_ERR_CUDA (-8)        /* a CUDA runtime call failed */
#define BF_ERR_UNSUPPORTED (-9) /* parameters outside what the kernels handle */
#define BF_ERR_BOUNDS (-10)     /* a device-side index check failed (checked build only) */

#define BF_MAX_D 8        /* channels per pixel */
#define BF_MAX_RADIUS 32  /* window half-width r of the windowed variants (sigma_s up to 10.99) */
#define BF_MAX_PLAN_RADIUS 4096 /* r of a plan (sigma_s up to 1365.6); beyond BF_MAX_RADIUS only
                                   BF_FP32_RECURSIVE filters with it */
#define BF_MAX_N 4096     /* raised-cosine order */
#define BF_MAX_K 65536    /* Monte Carlo terms */

/* Kernel variants of the blur step. */
#define BF_FP32 0   /* every step in FP32 on the CUDA cores */
#define BF_FP16TC 1 /* modulated channels in FP16, blur on tensor cores, FP32 accumulation */
#define BF_BF16TC 2 /* as BF_FP16TC with BF16 channels */
#define BF_FP32_RECURSIVE 3 /* FP32, the blur is Deriche's recursive Gaussian over the whole image
                               (O(1) in sigma_s, Section 3): a different filter from the 3-sigma
                               window (infinite support, ~1e-3 fit error); see bf_filter */

/* Whitening of the range kernel (Eq. COB). */
#define BF_WHITEN_CHOLESKY 0 /* W = L^{-1}, C = L L^T */
#define BF_WHITEN_EIGEN 1    /* W = diag(alpha) Q^T, C^{-1} = Q diag(alpha^2) Q^T (the paper's) */

typedef struct bf_plan_s *bf_plan_t; /* opaque; owned by the library */

/*
 * bf_plan -- build the sampled frequency list for (d, C, sigma_s, N, K, seed).
 * Follows Algorithm 1's set-up (diagonalise/whiten C, set up the spatial
 * filter, gamma = 1/sqrt(N)) and its "Draw X from B(N,1/2)^d" step, done once
 * for all K terms (Prop. 2, Eq. finalApproxY).
 *   d        channels, 1..BF_MAX_D (else BF_ERR_D_RANGE).
 *   C        host pointer, d*d doubles, row-major; symmetric positive definite
 *            (else BF_ERR_NOT_SPD; asymmetry beyond 1e-9 relative is BF_ERR_ARG).
 *   sigma_s  spatial standard deviation > 0; r = floor(3 sigma_s) must be
 *            <= BF_MAX_PLAN_RADIUS (else BF_ERR_UNSUPPORTED); the windowed
 *            variants further need r <= BF_MAX_RADIUS at filter time.
 *   N        raised-cosine order, 1..BF_MAX_N; 0 selects 10, the order used
 *            in all of the paper's experiments.
 *   K        Monte Carlo terms (the paper's T), 1..BF_MAX_K.
 *   seed     64-bit seed of the counter-based SplitMix64 stream: X_tk is the
 *            number of ones among N bits taken from ceil(N/64) consecutive
 *            outputs, t-major then k.
 *   out      receives the plan handle.
 * The whitening and the frequency vectors nu_t are computed on the device in
 * FP64 (Cholesky factor of C and back substitution); the call returns after
 * that kernel has finished.  The plan's device memory stays resident until
 * bf_plan_destroy.  Thread-safe; uses its own stream internally.
 */
int bf_plan(int d, const double *C, double sigma_s, int N, int K, uint64_t seed, bf_plan_t *out);

/* As bf_plan, with the whitening chosen by `whiten` (BF_WHITEN_*) and the
 * window half-width forced to `radius` when radius >= 0 (radius < 0 keeps
 * floor(3 sigma_s)). */
int bf_plan_ex(int d, const double *C, double sigma_s, int N, int K, uint64_t seed, int whiten, int radius,
               bf_plan_t *out);

/* Copy the plan's frequency list to host memory: nu_host (may be NULL) gets
 * K*d doubles, nu_t in turns (omega_t / 2 pi), row t = term; Y_host (may be
 * NULL) gets the K*d sampled integers Y_t = N - 2 X_t. */
int bf_plan_get_freqs(bf_plan_t plan, double *nu_host, int32_t *Y_host);

/* Plan parameters; any output pointer may be NULL. */
int bf_plan_info(bf_plan_t plan, int *d, int *K, int *N, int *radius, double *sigma_s);

/* Release the plan's device memory.  The caller must ensure no filtering call
 * that uses the plan is still in flight. */
int bf_plan_destroy(bf_plan_t plan);

/*
 * bf_filter -- apply the plan to one image (Algorithm 1's loop over t and the
 * final division), asynchronously on `stream`.
 *   in, out  device pointers, planar [d][H][pitch] FP32, 16-byte aligned
 *            (else BF_ERR_ALIGN); out receives S_c = Re P_c / Re Z for every
 *            pixel; padding columns x >= W of out are not written.
 *   H, W     image size; H == 0 or W == 0 is a no-op returning BF_OK.
 *   pitch    row stride in elements, pitch >= W and pitch % 4 == 0.
 *   variant  BF_FP32, BF_FP16TC, BF_BF16TC (windowed: r <= BF_MAX_RADIUS, else
 *            BF_ERR_UNSUPPORTED; the tensor-core variants need d = 3 or 6,
 *            else BF_ERR_UNSUPPORTED) or BF_FP32_RECURSIVE (any r; H <= 65535).
 *            With d = 6 the tensor-core kernel holds the image as 16-bit codes
 *            of a per-image affine map of each channel (error <= (max - min) /
 *            65535 of that channel, far below the FP16/BF16 channel rounding)
 *            and runs each term as two 8-channel passes.
 * Pixels whose Re Z is exactly 0 come out as IEEE inf/nan; nothing is clamped.
 * BF_FP32_RECURSIVE runs two kernels per term over the whole image and keeps
 * 2 x 2(d+1) + (d+1) FP32 planes of scratch per call in library memory.
 */
int bf_filter(bf_plan_t plan, const float *in, float *out, int H, int W, int pitch, int variant, void *stream);

/* One image of a batch. */
typedef struct {
    bf_plan_t plan;
    const float *in; /* device, planar [d][H][pitch] */
    float *out;      /* device, planar [d][H][pitch] */
    int H, W, pitch;
} bf_item;

/*
 * bf_filter_batch -- filter n independent images (each with its own plan,
 * size, d, sigma_s and K).  Tensor-core variants: one persistent-kernel launch
 * that pops tiles of all images from a device work queue (one for the d = 3
 * images, then one for the d = 6 images, preceded by a small kernel that
 * finds each six-channel image's per-channel range).  BF_FP32: one
 * launch per image, spread over 4 library-owned streams that are ordered
 * after the work already on `stream` and before anything queued on it later
 * (images run concurrently).  BF_FP32_RECURSIVE: one image after another on
 * `stream`.  Same rules per item as bf_filter; results equal those of n
 * separate bf_filter calls with the same variant.  `items` is a host array;
 * it is read before the call returns.
 */
int bf_filter_batch(const bf_item *items, int n, int variant, void *stream);

/*
 * bf_filter_batch_noalloc -- bf_filter_batch for the tensor-core variants that
 * allocates nothing.  The paper has no counterpart: this is a service of the
 * library, not a step of the method.
 *
 * bf_filter_batch and bf_filter keep their tile counter and image table in
 * device scratch that the library allocates (cudaMalloc) the first time a
 * stream needs it, or when a larger batch arrives.  Some callers cannot let a
 * library allocate: applications whose device memory is handed out entirely
 * by their own allocator (a framework's caching allocator, a fixed pool sized
 * at start-up), where a foreign cudaMalloc can fail or fragment the pool, and
 * latency-critical loops that cannot absorb the device-wide synchronisation a
 * cudaMalloc or cudaFree may cause.  This entry point serves them: its
 * scratch is a file-scope device array of 40.25 KB (the control words plus
 * the table and the six-channel range keys for BF_NOALLOC_MAX_ITEMS images) that every GPU loading the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree or
 * other allocating routine, on the device or the host.
 *   items, stream   as bf_filter_batch; the caller still owns every image.
 *   variant         BF_FP16TC or BF_BF16TC (else BF_ERR_ARG); every image
 *                   must have d = 3 or 6 (else BF_ERR_UNSUPPORTED).
 *   n               0..BF_NOALLOC_MAX_ITEMS; larger n returns BF_ERR_BUDGET
 *                   before any work is queued (split the batch).
 * Results are identical to bf_filter_batch with the same arguments.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current) and caches it.  The call
 * uploads its table from host memory of the call itself, so it returns
 * BF_ERR_ARG on a stream that is being captured.  All calls share the one array and
 * it keeps the last call's contents: each call resets the tile counter and
 * rewrites the table, so calls whose work overlaps on the GPU (on different
 * streams, or from several host threads) race and must be serialised by the
 * caller.  Timeouts recorded by its kernel are reported by bf_last_status.
 */
#define BF_NOALLOC_MAX_ITEMS 256
int bf_filter_batch_noalloc(const bf_item *items, int n, int variant, void *stream);

/*
 * Tuning of the windowed kernels' tile height.  The paper has no counterpart:
 * it is a service of the library (the batched and served forms pick their
 * tiles from measurements; the paper's own Table 1 axis is sigma_s, i.e. r).
 *
 * The tile height (output rows per CTA tile, a multiple of 16) of the
 * BF_FP32, BF_FP16TC and BF_BF16TC kernels changes no result, only how the
 * work spreads over the SMs and how much of the r-pixel halo each tile
 * recomputes.  Without an entry a launch uses its cost model (tile waves x
 * steps per tile for an image alone, the tallest tile in a batch).  Entries
 * are keyed by (variant, d, radius class, size class, context):
 *   radius class ceil(r / 8): r = 0, 1..8, 9..16, 17..24, 25..32 (the classes
 *                share the tensor-core tile geometry); set or get with any r
 *                of the class
 *   size class   bf_tune_size_class(H, W) = 32 floor(2 log2 H) + floor(2 log2 W)
 *                (half-octave classes of height and width)
 *   context      BF_TUNE_ALONE: the image is the only one of its launch
 *                (bf_filter, a batch of one); BF_TUNE_BATCH: one of several
 *                images of one persistent launch (or of the forked FP32 batch)
 *   tile_rows    16..128 in steps of 16; a launch clamps it to what its
 *                window and shared memory allow; 0 removes the entry
 * The table is process-wide and thread-safe; tune.py fills it from timings
 * and keeps a JSON cache.  Returns BF_OK or BF_ERR_ARG (bad key or value).
 */
#define BF_TUNE_ALONE 0
#define BF_TUNE_BATCH 1
int bf_tune_size_class(int H, int W); /* the class, or BF_ERR_ARG for H or W <= 0 */
int bf_tune_set(int variant, int d, int r, int size_class, int context, int tile_rows);
int bf_tune_get(int variant, int d, int r, int size_class, int context, int *tile_rows); /* 0: none */
int bf_tune_clear(void);
int bf_tune_count(void); /* number of entries */

/*
 * bf_filter_host -- end-to-end convenience call for callers holding host
 * images: copies `in_host` (planar [d][H][W], pitch W) to library-owned
 * device buffers, filters, copies the result to `out_host`, and synchronises
 * `stream` before returning.  Host buffers may be pageable; pinned buffers
 * give overlapped copies.  The device buffers are cached per library and
 * grown on demand (BF_ERR_NOMEM if that fails).  Not re-entrant on the same
 * stream from several host threads.
 */
int bf_filter_host(bf_plan_t plan, const float *in_host, float *out_host, int H, int W, int variant,
                   void *stream);

/*
 * bf_rgb_to_lab / bf_lab_to_rgb -- colour transforms for filtering in CIE-Lab,
 * as the paper does for its House example (Section 4, Fig. 4): convert, filter
 * the Lab image with a plan whose C is in Lab units, convert back.
 * The RGB side is sRGB on the 0..255 scale (IEC 61966-2-1 transfer function
 * and D65 matrix), the Lab side CIE 1976 (L*, a*, b*) with the white point of
 * RGB white; nothing is clipped in either direction.
 *   in, out  device pointers, planar [3][H][pitch] FP32, 16-byte aligned
 *            (else BF_ERR_ALIGN); in == out (in place) is allowed, any other
 *            overlap is BF_ERR_ARG.
 *   H, W     image size (0 is a no-op); pitch >= W, pitch % 4 == 0.
 * Asynchronous on `stream`; one elementwise kernel each.
 */
int bf_rgb_to_lab(const float *in, float *out, int H, int W, int pitch, void *stream);
int bf_lab_to_rgb(const float *in, float *out, int H, int W, int pitch, void *stream);

/*
 * bf_filter_host_async -- bf_filter_host without the final synchronisation:
 * the copy in, the filter and the copy out are queued on `stream` and the call
 * returns.  For the copies to be asynchronous the host buffers must be pinned
 * (cudaHostAlloc / cudaHostRegister); they must stay valid, and out_host must
 * not be read, until the stream has reached this work (synchronise it or wait
 * on an event recorded after the call).  Device buffers are per (device,
 * stream), kept by the library and reused by the next call on the same stream,
 * which the stream orders after this one; calls on different streams overlap
 * (the copies of one with the filter of another).
 */
int bf_filter_host_async(bf_plan_t plan, const float *in_host, float *out_host, int H, int W, int variant,
                         void *stream);

/* Status word of the library's device-side guards (bounded waits, tile-queue
 * consistency) for work issued on `stream`; synchronises the stream, returns
 * BF_OK or the first BF_ERR_* recorded, and clears it. */
int bf_last_status(void *stream);

/* Fault injection, for tests of the error paths (no fault, trap or hang is
 * ever caused on the device).  Arms one-shot faults, OR-ed into those already
 * armed (0 disarms all); each is consumed by the first call that reaches it:
 *   BF_FAULT_ALLOC    the next request to the library's device allocators
 *                     (plan creation, per-stream scratch) fails with
 *                     BF_ERR_NOMEM, as if the device were out of memory;
 *   BF_FAULT_TC_WAIT  the next tensor-core launch skips its first group of
 *                     MMAs and uses a short spin limit, so the compute warps'
 *                     bounded wait runs out: every CTA stops after its first
 *                     tile, the output is not written, the launch's status
 *                     word reads BF_ERR_TIMEOUT (bf_last_status).
 * Returns BF_OK, or BF_ERR_ARG for an unknown bit.  Thread-safe. */
#define BF_FAULT_ALLOC 1
#define BF_FAULT_TC_WAIT 2
int bf_debug_inject(int faults);

/* Static description of an error code. */
const char *bf_error_string(int code);

/* Library version, e.g. 10000 for 1.0.0. */
int bf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BF_H_ */
