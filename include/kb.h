/*
 * kb.h -- C ABI of the GB300 (sm_103a) shift-and-stack likelihood search.
 *
 * The method is the one of Whidden et al., "Fast algorithms for slow moving
 * asteroids" (arXiv:1901.02492):
 *   stage (a)  per epoch t, the likelihood images of Sec. 2.1.5
 *                psi_t(y) = sum_i n_t(x_i) T_t(x_i - y) / sigma_t,i^2
 *                phi_t(y) = sum_i T_t(x_i - y)^2 / sigma_t,i^2
 *              with masked pixels given zero inverse variance (Sec. 2.1.5);
 *   stage (b)  for every start pixel y0 of the earliest image and every velocity
 *              v of a grid (Sec. 2.2, Sec. 3.2), the coadd of Sec. 2.1.5
 *                Psi = sum_t psi_t(y0 + v t),  Phi = sum_t phi_t(y0 + v t),
 *              the scores alpha = Psi / Phi (maxLikeFlux) and nu = Psi / sqrt(Phi),
 *              keeping the k best trajectories per start pixel.
 *
 * Conventions shared by every call:
 *   - Images are row-major [N][H][W] (epoch, row y, column x); a trajectory
 *     pixel is (x0 + dx, y0 + dy).
 *   - "device pointer" means memory of the context's CUDA device (cudaMalloc,
 *     torch CUDA tensors, ...); "host pointer" means ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is stream-ordered: inputs must stay valid until the stream has
 *     executed the call's work; outputs are ready when it has.
 *   - Every call returns KB_OK (0) or a KB_E* status; no exception crosses the
 *     ABI.  The text of the last error of a context is kb_last_error(ctx).
 *   - A context, and the stacks and jobs made from it, are used from one host
 *     thread at a time.
 *
 * Trajectory pixels are computed in fixed point, identically for every call
 * (the paper rounds y0 + v t to a pixel without saying how):
 *   v_q = llround(v * 2^16)                  (v in px/day)
 *   t_q = llround((t - t_min) * 2^20)        (t in days, t_min = earliest epoch)
 *   d   = floor((v_q * t_q + 2^35) / 2^36)   (64-bit integers; round half up)
 * so |v| < 2^12 px/day and t - t_min < 2^6 days are required.
 */
#ifndef KB_H
#define KB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define KB_OK 0
#define KB_EINVAL 1   /* bad argument: NULL pointer, bad shape or size, K even, ... */
#define KB_ENOMEM 2   /* device allocation failed or the context's HBM budget is exceeded */
#define KB_ECUDA 3    /* a CUDA runtime call failed (message in kb_last_error) */
#define KB_ETIMEOUT 4 /* a bounded device-side wait gave up */
#define KB_ERANGE 5   /* output buffer too small; *n_written holds the required count */

/* ---- storage of the psi/phi planes used by the search ------------------- */
#define KB_F32 0   /* (psi, phi) as two float32 per pixel, 8 bytes */
#define KB_BF16 1  /* (psi, phi) as two bfloat16 per pixel with per-epoch power-of-two scales, 4 bytes */
#define KB_F16 2   /* (psi, phi) as two float16 per pixel with per-epoch power-of-two scales, 4 bytes */

/* ---- search flags -------------------------------------------------------- */
#define KB_RESCORE_FP64 1 /* re-rank the kept candidates with FP64 sums of the FP32 planes;
                           * pixels the certificate cannot clear are re-searched in FP64 */
#define KB_PRUNE 2        /* kb_search with nu_min > 0: skip the gathers of a warp's span of
                           * start pixels for a velocity when a bound on nu over the span
                           * cannot reach nu_min (Sec. 5.3); the results are unchanged */

/* ---- limits -------------------------------------------------------------- */
#define KB_MAX_EPOCHS 128   /* N */
#define KB_MAX_PSF 63       /* K (odd) */
#define KB_MAX_TOPK 16      /* k */
#define KB_MAX_VELOCITIES 65535
#define KB_MAX_SIDE 32767   /* H and W */

typedef struct kb_ctx kb_ctx;     /* one CUDA device, an HBM budget, the last error */
typedef struct kb_stack kb_stack; /* device-resident psi/phi planes of one image stack */
typedef struct kb_job kb_job;     /* device-resident results of one search */

/* One kept trajectory (Sec. 2.2), as written by kb_results (48 bytes). */
typedef struct kb_result {
    int32_t x0, y0;   /* start pixel in the earliest epoch (column, row) */
    int32_t vidx;     /* index into the caller's velocity arrays; -1 = empty slot */
    int32_t nobs;     /* epochs whose trajectory pixel lies inside the image */
    float vx, vy;     /* the velocity as quantised by the library, px/day (v_q / 2^16) */
    float psi, phi;   /* coadded Psi and Phi (Sec. 2.1.5) */
    double nu, alpha; /* nu = Psi / sqrt(Phi), alpha = Psi / Phi; empty slot: nu = -inf, alpha = 0 */
} kb_result;

/* ---- context ------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps what the
 * context's stacks and jobs may hold on the device (0 = no cap); allocations
 * beyond it fail with KB_ENOMEM.  Device memory comes from a stream-ordered
 * pool of the context, so creating and freeing stacks and jobs never waits for
 * kernels running on other streams; freed blocks stay in the pool for reuse
 * until kb_destroy.  *ctx is owned by the caller: kb_destroy. */
int kb_init(kb_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Free the context.  Stacks and jobs made from it must be freed first. */
void kb_destroy(kb_ctx *ctx);

/* NUL-terminated text of the context's last error ("" if none); owned by ctx. */
const char *kb_last_error(const kb_ctx *ctx);

/* Bytes of device memory currently held by the context's stacks and jobs. */
size_t kb_hbm_in_use(const kb_ctx *ctx);

/* Bounds words of a KB_DEBUG build (libkb_debug.so, built by
 * paper_1901_02492_gb300.build.build(debug=True)).  In such a build every gather
 * of the search kernels from the psi/phi planes, every write of their offset
 * tables in shared memory and every list column they insert into is checked
 * against its extent; an access outside is skipped (a gather reads zero) and the
 * first one since the last reset is recorded, never trapped.
 * kb_debug_build: 1 in a KB_DEBUG build, 0 otherwise.
 * kb_debug_word: *word = (site << 56) | offset of that first access (0 if none;
 * sites: 1 reference-epoch gather, 2 batched gather, 3 remainder gather,
 * 4 predicated gather, byte offsets from the planes' base; 5 table entry,
 * 6 list column, element indices); reset != 0 clears it afterwards.  It
 * synchronises the device.  KB_EINVAL in a build without KB_DEBUG or for a
 * NULL argument. */
int kb_debug_build(void);
int kb_debug_word(kb_ctx *ctx, unsigned long long *word, int reset);

/* Tuning hook: force the search kernel used by later kb_search calls of this
 * context; results do not depend on the choice.
 *   0      automatic: the register-gather kernel in its default shape, (2,8) for
 *          FP32 and (2,4) for 16-bit storage ((1,4) for value lists longer than 8)
 *   1..4   register-gather kernel, (loads per lane, epochs per load batch) =
 *          (4,4), (2,4), (4,8), (2,8) for FP32 and (2,4), (1,4), (2,8), (1,8)
 *          for 16-bit storage, whose loads are pixel pairs
 *   5..8   TMA-pipelined kernel, (pixels per lane, stages, epochs per wait
 *          group) = (2,8,2), (2,12,4), (4,8,2), (4,12,4)
 * KB_EINVAL for other values. */
int kb_set_search_variant(kb_ctx *ctx, int variant);

/* Tuning hook: preferred shared-memory carveout of the register-gather search
 * kernel, in percent of the maximum (cudaFuncAttributePreferredSharedMemoryCarveout);
 * -1 = automatic.  It trades resident CTAs against L1 capacity, which the
 * gathers of the early epochs reuse.  Results do not depend on it. */
int kb_set_search_carveout(kb_ctx *ctx, int percent);

/* Tuning knob: the order in which the register-gather search kernel's CTAs
 * take their start-pixel tiles.  cols > 0: the tiles are dealt out in
 * super-columns `cols` tiles wide, row by row within each (so the CTAs resident
 * at one time cover a block about cols tiles wide instead of whole rows of
 * tiles); 0: row by row over the whole image; -1: automatic, which is 8.  The
 * late epochs' rows that a resident block reads then stay in L2: on the
 * 12 x 4096^2 stack (64 tiles per row) the FP32 search takes 97.7 ms with 8
 * against 117.4 ms row by row.  Results do not depend on it. */
int kb_set_search_swizzle(kb_ctx *ctx, int cols);

/* Tuning knob: the order in which every CTA of the search walks the velocities.
 * 0: by the trajectory offset at the latest epoch, dy then dx; 1: along a
 * Hilbert curve over those offsets (velocities walked close together are close
 * in both axes); 2: the caller's order; -1: automatic (0).  On the
 * 12 x 4096^2 stack: 97.7, 102.5 and 98.7 ms.  Ties in nu are broken by the
 * caller's velocity index, so results do not depend on it. */
int kb_set_search_order(kb_ctx *ctx, int order);

/* Measurement helper (no counterpart in the paper): the L2-to-SM bandwidth, in
 * GB/s, of the search's own access form -- each warp reads warp_bytes (256, 512
 * or 1024) contiguous bytes as lane-contiguous 8-byte loads, starting at a
 * scattered multiple of align_bytes (a power of two >= 8; 8 is the search's
 * form, whose shifted spans start at any pixel) of an L2-resident 64 MB buffer,
 * from every SM, not cached in L1.  It is the denominator of the search's
 * roofline.  Takes about 100 ms; allocates and frees 64 MB on the context's
 * device.  KB_EINVAL for other sizes. */
int kb_measure_gather_peak(kb_ctx *ctx, int warp_bytes, int align_bytes, double *gb_per_s);

/* ---- stage (a): likelihood images --------------------------------------- */

/* Allocate the device planes for an N x H x W stack (1 <= N <= KB_MAX_EPOCHS,
 * 1 <= H, W <= KB_MAX_SIDE).  The FP32 (psi, phi) planes are always kept; with
 * storage KB_BF16 or KB_F16 a 16-bit copy with per-epoch scales is kept as well
 * (twice: also shifted by one pixel, so that any two adjacent pixels are one
 * aligned load) and is what kb_search reads.  Device memory: N * (H + 16) * (W + 260)
 * * 8 bytes, twice that with 16-bit storage.  *out is owned by the caller:
 * kb_stack_free. */
int kb_stack_create(kb_ctx *ctx, int N, int H, int W, int storage, kb_stack **out);
/* Release the stack.  Its memory is reused only after the last kb_make_psi_phi,
 * kb_search or kb_stack_copy_planes on it has finished on the device; when the
 * stack was searched from several streams at once, the caller waits for all of
 * them first.  Does not block on kernels of other stacks. */
void kb_stack_free(kb_stack *s);

/* Sec. 2.1.5: fill the stack with psi_t and phi_t of every epoch.
 *   sci   device, float [N][H][W]: background-subtracted counts n(x)
 *   var   device, float [N][H][W]: variance sigma^2
 *   mask  device, uint8 [N][H][W] or NULL: non-zero = masked
 *   psf   HOST, float [N][K][K]: PSF T_t of each epoch, row-major, T(dy, dx) at
 *         [(dy + K/2) * K + (dx + K/2)]; K odd, 1 <= K <= KB_MAX_PSF.  Separable
 *         (rank-1) kernels take a two-pass path, others a single-pass 2-D path.
 *   bright_max  pixels with n > bright_max are masked (Sec. 5.2); pass +inf or
 *         NaN to disable.
 * A pixel is masked when its mask byte is non-zero, when n or sigma^2 is not
 * finite, when sigma^2 <= 0, or when n > bright_max; it then contributes exactly
 * zero.  PSF taps falling outside the image contribute zero.  The psf array is
 * read before the call returns; the device inputs are read in stream order. */
int kb_make_psi_phi(kb_stack *s, const float *sci, const float *var, const uint8_t *mask, const float *psf,
                    int K, float bright_max, void *stream);

/* The likelihood images of kb_make_psi_phi without allocating anything.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory where they need the planes -- code whose device
 * memory belongs to another allocator, or loops in which cudaMalloc/cudaFree
 * are not allowed because they can block or synchronise the device.
 *   sci, var  device, float [N][H][W]; mask device uint8 [N][H][W] or NULL
 *   psf       HOST, float [N][K][K], as for kb_make_psi_phi
 *   out       device, float [N][H][W][2]: (psi, phi) per pixel, caller-owned
 * Same arithmetic and results as kb_make_psi_phi followed by
 * kb_stack_copy_planes(which = 0).  Works on the calling thread's current
 * device and in stream order.  The per-epoch PSF taps it needs are kept in a
 * static device array of 256 KB (65536 floats) that every GPU loading the
 * library holds until exit: separable PSFs need N * 4K floats, other PSFs
 * N * 2K^2 floats, and a call that needs more returns KB_EINVAL.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing).  The taps are staged through
 * one host buffer that every call rewrites, so a call on a stream that is being
 * captured into a CUDA graph is refused with KB_EINVAL before any other work: a
 * captured copy would read the buffer at replay, after other calls changed it.
 * All calls share the array, so calls that overlap on the GPU (e.g. on
 * different streams) race and must be ordered by the caller.  The library
 * cannot check the sizes of the caller's buffers: sci, var (and mask) must hold
 * N*H*W elements and out 2*N*H*W floats.  Returns KB_OK, KB_EINVAL (bad sizes
 * or pointers, too many taps, or a capturing stream) or KB_ECUDA. */
int kb_make_psi_phi_static(const float *sci, const float *var, const uint8_t *mask, const float *psf, int N, int H,
                           int W, int K, float bright_max, float *out, void *stream);

/* Copy the stack's planes to dst (host or device), stream-ordered.
 *   which = 0: FP32 planes, float [N][H][W][2] = (psi, phi), dst_bytes >= N*H*W*8
 *   which = 1: 16-bit planes, uint16 [N][H][W][2] = (psi, phi) codes, dst_bytes >= N*H*W*4
 *              (value = code * scale of that epoch, see kb_stack_scales)
 *   which = 2: the span bound planes of the last KB_PRUNE search, float
 *              [N][H][(W + 31) / 32 + span / 32] (entry c + span / 32: the
 *              largest max(psi, 0)^2 / phi over the image columns
 *              [32 c, 32 c + span + 32)), dst_bytes >= their size; KB_EINVAL if
 *              none are built
 * Host destinations make the call synchronous.  KB_EINVAL if the stack has no
 * such planes or dst_bytes is too small. */
int kb_stack_copy_planes(const kb_stack *s, int which, void *dst, size_t dst_bytes, void *stream);

/* Per-epoch power-of-two scales of the 16-bit planes (host arrays of N floats);
 * synchronises with the work that made them.  All 1.0 for KB_F32 stacks. */
int kb_stack_scales(const kb_stack *s, float *psi_scale, float *phi_scale);

/* ---- stage (b): trajectory search ---------------------------------------- */

/* The trajectory offsets the search uses, in the fixed point defined above:
 * dx, dy host int32 [V][N] for the caller's epoch order.  times host [N] days,
 * vx, vy host [V] px/day.  Pure host function. */
int kb_offsets(const double *times, int N, const double *vx, const double *vy, int V, int32_t *dx,
               int32_t *dy);

/* Allocate a search job for H x W start pixels, up to N epochs, up to V
 * velocities and up to topk results per pixel (1 <= topk <= KB_MAX_TOPK).
 * flags may include KB_RESCORE_FP64 (reserves the candidate buffers).
 * *out is owned by the caller: kb_job_free. */
int kb_job_create(kb_ctx *ctx, int H, int W, int N, int V, int topk, int flags, kb_job **out);
/* Release the job; its memory is reused only after its last search finished. */
void kb_job_free(kb_job *j);

/* Sec. 2.2 exhaustive search of the stack s into job:
 *   times   host double [N]: epoch times in days, in the stack's epoch order
 *   vx, vy  host double [V]: velocity grid in px/day (the caller's index = vidx)
 *   topk    results kept per start pixel (<= the job's topk)
 *   nu_min  only trajectories with nu >= nu_min are kept (-inf keeps all valid)
 *   flags   KB_RESCORE_FP64: search the stack's planes keeping extra
 *           candidates, then recompute each candidate's sums in FP64 from the
 *           FP32 planes, re-rank in FP64 and keep the top-k.
 *           KB_PRUNE (with nu_min > 0 and the automatic kernel shape): by
 *           Cauchy-Schwarz, nu^2 <= sum_t max(psi_t, 0)^2 / phi_t over a
 *           trajectory's in-image epochs; per epoch and row the largest such
 *           term over windows [32 c, 32 c + span + 32) that cover a warp span of
 *           the shifted start pixels is precomputed (a stack cache of
 *           N * H * ((W + 31) / 32 + span / 32) floats, span = 64 or 128 pixels
 *           by storage and k, allocated under the budget and rebuilt after
 *           kb_make_psi_phi), and a velocity whose span bound
 *           (rounded upwards, with a 2^-14 relative margin) is below nu_min^2 is
 *           skipped for that span.  The records equal those of the same search
 *           without the flag, byte for byte.  Ignored otherwise (and by batches).
 * Every start pixel of the earliest epoch is searched.  Epochs whose trajectory
 * pixel is outside the image contribute nothing; trajectories with Phi == 0 are
 * not kept; ranking is by (nu descending, vidx ascending); empty slots have
 * vidx = -1.  The host arrays are read before the call returns; the kernels run
 * in stream order and may be re-run by calling kb_search again. */
int kb_search(kb_job *job, const kb_stack *s, const double *times, const double *vx, const double *vy, int V,
              int topk, float nu_min, int flags, void *stream);

/* Wait for the job's last search and report its device status: KB_OK, or
 * KB_ETIMEOUT when a bounded device-side wait of the pipelined kernel gave up
 * (its results are then invalid).  kb_results with a host destination calls it. */
int kb_job_wait(kb_job *job);

/* After a search with KB_RESCORE_FP64: the number of start pixels whose
 * rescored top-k the certificate could not clear and that were searched again
 * exhaustively in FP64 (waits for the job like kb_job_wait).  The certificate:
 * a trajectory outside the k_c candidates of the reduced-precision pass scored
 * at most nu16 of the last candidate; the pixel is cleared when the k-th FP64
 * nu (or nu_min) exceeds that by more than twice the largest |nu16 - nu64| of
 * the pixel's own candidates plus the storage unit roundoff times (1 + |nu|).
 * 0 for searches without rescoring. */
int kb_job_repaired(kb_job *job, size_t *n_pixels);

/* Write the job's results as kb_result records, [H][W][topk] in start-pixel
 * row-major order, best first within a pixel.  out is a host or device pointer
 * with room for `capacity` records; a host destination makes the call wait for
 * the stream (host records go through device staging in chunks of 2^22 and
 * copies).  KB_ERANGE (with *n_written = H*W*topk) if capacity is too small. */
int kb_results(kb_job *job, kb_result *out, size_t capacity, size_t *n_written, void *stream);

/* kb_results without any host wait: the expansion and the copies are enqueued
 * on `stream` (which first waits for the job's last search), and the call
 * returns.  A host destination is served by one expansion into job-owned
 * device staging of H*W*topk records (allocated on first use, under the HBM
 * budget) and one copy, so that after the short expansion only the copy engine
 * works and the copy overlaps later kernels.  out must be device memory or page-locked host memory
 * (cudaMallocHost / cudaHostRegister), else KB_EINVAL; it is complete once
 * `stream` has reached this point.  A later kb_search or kb_batch_run of the
 * job, and kb_job_free, wait on the device for the read to finish, so results
 * of one job can be copied out while another job searches.  The search's
 * device status is read with kb_job_wait. */
int kb_results_async(kb_job *job, kb_result *out, size_t capacity, size_t *n_written, void *stream);

/* One kept trajectory in 16 bytes, as written by kb_results_compact_async: the
 * fields of kb_result that cannot be derived from the record's position
 * ([H][W][topk], row-major start pixels, best first) and the caller's velocity
 * grid.  Little-endian layout; static_assert-checked against the search's own
 * device record. */
typedef struct kb_result_compact {
    float psi, phi;   /* coadded Psi and Phi (Sec. 2.1.5); FP64 values rounded to FP32 after rescoring */
    float nu;         /* Psi / sqrt(Phi) as ranked (rounded to FP32 after rescoring); -inf when empty */
    uint16_t vidx;    /* index into the caller's velocity arrays; 0xFFFF = empty slot */
    uint8_t nobs;     /* epochs whose trajectory pixel lies inside the image */
    uint8_t reserved; /* 0 */
} kb_result_compact;

/* kb_results_async with compact records (not a step of the paper: a transfer
 * format).  Writes H*W*topk kb_result_compact records into out (device or
 * page-locked host memory), stream-ordered, without a host wait, and with the
 * ordering guarantees of kb_results_async.  A search without rescoring already
 * holds its records in this form on the device, so they are copied as they are
 * (one copy, no kernel): a third of the bytes of kb_result, which matters where
 * the records cross the host link every step.  Rescored jobs convert their FP64
 * records with one kernel first (through job-owned staging for host
 * destinations).  KB_ERANGE (with *n_written = H*W*topk) if capacity (in
 * records) is too small; KB_EINVAL for pageable host memory. */
int kb_results_compact_async(kb_job *job, kb_result_compact *out, size_t capacity, size_t *n_written,
                             void *stream);

/* ---- light-curve outlier filter of kept trajectories (Sec. 3.3) ---------- */

/* One filtered trajectory (72 bytes). */
typedef struct kb_filtered {
    int32_t x0, y0;        /* start pixel */
    int32_t vidx;          /* velocity index as in kb_results; -1 = empty slot */
    int32_t nobs;          /* epochs kept: trajectory pixel in the image, not rejected */
    int32_t nrejected;     /* epochs rejected as outliers */
    int32_t reserved;
    uint32_t rejected[4];  /* bit e % 32 of word e / 32: stack epoch e rejected */
    double psi, phi;       /* coadd over the kept epochs, FP64 sums of the FP32 planes */
    double nu, alpha;      /* psi / sqrt(phi), psi / phi; -inf and 0 when phi == 0 or empty */
} kb_filtered;

/* Sec. 3.3: for every kept trajectory of the job's last search (H*W*topk of
 * them, the records kb_results would write), reject the observations that lie
 * more than `nsigma` standard deviations from the best-fit flux of the others
 * and recompute the likelihood from the rest.  Reading of the paper's Kalman
 * variant: the flux is constant, so the estimate from a set of observations is
 * their inverse-variance weighted mean; epoch e (pixel in the image, phi_e > 0)
 * with flux psi_e / phi_e is rejected when it differs from the others' estimate
 * (Psi - psi_e) / (Phi - phi_e) by more than nsigma sqrt(1 / phi_e + 1 / (Phi -
 * phi_e)), all decisions on the unfiltered sums, in FP64.
 *   s      the stack that was searched (its FP32 planes are read)
 *   out    DEVICE pointer, room for `capacity` records, written [H][W][topk]
 * KB_EINVAL (no search yet, stack shape differs, nsigma <= 0, out not device
 * memory), KB_ERANGE (capacity < H*W*topk; *n_written says how many).  Runs in
 * stream order after the search. */
int kb_filter_lightcurves(kb_job *job, const kb_stack *s, double nsigma, kb_filtered *out, size_t capacity,
                          size_t *n_written, void *stream);

/* ---- coadded postage stamps and central moments (Sec. 3.3) --------------- */

#define KB_STAMP_MEAN 0
#define KB_STAMP_MEDIAN 1
#define KB_MAX_STAMP_RADIUS 15   /* stamps up to 31 x 31 */

/* Central moments of one coadded stamp (coordinates relative to its centre,
 * pixel values as weights) and the result of the Gaussian-similarity cut. */
typedef struct kb_moments {
    double m00;            /* sum of the stamp over the aperture */
    double mx, my;         /* centroid */
    double mu20, mu02, mu11; /* central second moments over m00 */
    int32_t passed;        /* 1: passed the cuts (or no cuts given), 0: rejected */
    int32_t reserved;
} kb_moments;

/* Cuts of the moment filter (moments over the aperture): a stamp passes when
 * m00 > 0, |mx|, |my| <= max_offset, min_var <= mu20, mu02 <= max_var and
 * |mu11| <= max_mu11.  The caller derives them from the epochs' PSF widths. */
typedef struct kb_moment_cuts {
    double max_offset, min_var, max_var, max_mu11;
} kb_moment_cuts;

/* Sec. 3.3: coadded postage stamps along candidate trajectories of the job's
 * last search.  For candidate i (start pixel (x0[i], y0[i]), velocity vidx[i]
 * of that search) and stamp pixel (sx, sy) in [-r, r]^2, the values of
 * sci[e][y0 + dy_e + sy][x0 + dx_e + sx] over the epochs e whose pixel is in
 * the image, finite and not masked, with the search's own trajectory offsets,
 * combined as their mean (KB_STAMP_MEAN, FP64 sum) or median (KB_STAMP_MEDIAN:
 * the middle value, the mean of the two middle ones for an even count); 0 where
 * no epoch contributes.  Then the stamp's central moments over the aperture
 * sx^2 + sy^2 <= aperture^2 (the whole stamp when aperture <= 0; about two PSF
 * widths keeps a faint source's light and little of the sky noise around it)
 * and, with `cuts`, the moment filter.
 *   sci, mask  DEVICE [N][H][W] science images (and mask or NULL), the job's N, H, W
 *   x0, y0, vidx  HOST [n] candidates
 *   stamps     DEVICE float [n][2r+1][2r+1]; moments DEVICE [n] or NULL
 * KB_EINVAL (no search yet, shapes, r outside 0..KB_MAX_STAMP_RADIUS, a NaN
 * aperture, a candidate outside the image or velocity range, pointers).
 * Stream-ordered; the host arrays are read before the call returns. */
int kb_stamps(kb_job *job, const float *sci, const uint8_t *mask, int N, int H, int W, const int32_t *x0,
              const int32_t *y0, const int32_t *vidx, int n, int radius, int mode, double aperture,
              const kb_moment_cuts *cuts, float *stamps, kb_moments *moments, void *stream);

/* ---- de-duplication of candidates (Sec. 3.3) ------------------------------ */

typedef struct kb_cluster_params {
    double w_pos;        /* weight of the start-pixel coordinates (1/px) */
    double w_vel;        /* weight of the velocity coordinates (day/px) */
    double eps;          /* neighbourhood radius in the weighted coordinates */
    int32_t min_samples; /* neighbours (the point included) that make a core point */
    int32_t reserved;
} kb_cluster_params;

/* Sec. 3.3: groups similar candidate trajectories with DBSCAN and keeps the
 * highest-likelihood trajectory of each group.  The distance between
 * candidates i and j is the Euclidean distance of (x0 w_pos, y0 w_pos,
 * vx w_vel, vy w_vel), evaluated in FP64 as
 *     d2 = ((ax*ax + ay*ay) + au*au) + av*av,
 *     ax = (double)(x0_i - x0_j) * w_pos (ay likewise),
 *     au = ((double)vx_i - (double)vx_j) * w_vel (av likewise),
 * every operation rounded (no fused multiply-add); j is a neighbour of i when
 * d2 <= eps*eps, i included.  Then:
 *   core point   at least min_samples neighbours;
 *   cluster      a connected component of core points under the neighbour
 *                relation, labelled by its lowest core index;
 *   border point a non-core point with a core neighbour: joins the cluster of
 *                its nearest core neighbour (smallest d2, then lowest index);
 *   noise point  a group of its own, labelled by its own index;
 *   vidx < 0     (an empty result slot) takes no part: label -1, keep 0.
 * keep[i] = 1 for the member of each group with the largest nu (then lowest
 * index).
 *   cand       DEVICE [n] kb_result records (e.g. from kb_results)
 *   label      DEVICE [n] int32; keep DEVICE [n] uint8; core DEVICE [n] or NULL
 *   n_groups   HOST, or NULL: the number of kept candidates
 * KB_EINVAL (n > 2^29, weights or eps not positive and finite, min_samples < 1,
 * pointers, or a weighted coordinate beyond 2^30 eps).  Stream-ordered on
 * `stream`; returns after the stream has finished the call's work. */
int kb_cluster(kb_ctx *ctx, const kb_result *cand, size_t n, const kb_cluster_params *p, int32_t *label,
               uint8_t *keep, uint8_t *core, size_t *n_groups, void *stream);

/* Device bytes that one search will hold, for admission under an HBM budget:
 *   *stack  kb_stack_create(N, H, W, storage) plus kb_make_psi_phi with a K x K
 *           PSF (an upper bound: the tap table of a non-separable PSF)
 *   *job    kb_job_create(H, W, N, V, topk, flags)
 * Not included: the staging that kb_results allocates on its first host-bound
 * call (at most 2^22 records, 192 MiB).  Either pointer may be NULL.  KB_EINVAL
 * for arguments that kb_stack_create or kb_job_create would reject. */
int kb_estimate_bytes(int N, int H, int W, int storage, int K, int V, int topk, int flags, size_t *stack,
                      size_t *job);

/* ---- batched searches (no counterpart in the paper: many stacks per launch) ----
 *
 * A batch runs many independent Sec. 2.2 searches, of stacks with different
 * sizes, epoch counts, velocity grids and k, grouped by storage, index width and
 * candidate-list length.  Each group runs with one of two schedules: one
 * persistent launch whose CTAs take items off a work list (one item per CTA tile
 * of every search, in order of per-tile cost, largest search first), or one
 * launch per search.  The launches, and the FP64 rescoring of the searches that
 * ask for it, are captured once into a CUDA graph that kb_batch_run replays.
 * Every search gives the results that kb_search gives for the same arguments
 * and tile shape. */
typedef struct kb_batch kb_batch;

/* One search of a batch: the arguments of kb_search (same meaning and limits). */
typedef struct kb_batch_item {
    kb_job *job;            /* distinct per item; holds the search's tables and results */
    const kb_stack *stack;
    const double *times;    /* host [stack N] */
    const double *vx, *vy;  /* host [V] */
    int V;
    int topk;
    float nu_min;
    int flags;              /* KB_RESCORE_FP64 or 0 */
} kb_batch_item;

#define KB_BATCH_AUTOTUNE 1 /* time every tile shape and schedule per group, keep the fastest */

/* The plan of one group (filled by kb_batch_groups). */
typedef struct kb_batch_group {
    int storage;            /* KB_F32 / KB_BF16 / KB_F16 */
    int index_bits;         /* 32 or 64: width of the element offsets */
    int variant;            /* tile shape 1..4 (see kb_set_search_variant) */
    int kmax;               /* candidate-list length of its searches */
    long long n_items;      /* CTA tiles in its work list */
    double evals;           /* trajectory-epoch evaluations of its searches */
    float tuned_ms[5];      /* autotuner time of shapes 1..4, persistent schedule, on its sample (0: not tuned) */
    int schedule;           /* 0: one persistent launch over the group's work list; 1: one launch per search */
    float tuned_ms_launch[5]; /* autotuner time of shapes 1..4 with one launch per search (0: not tuned) */
} kb_batch_group;

/* Validate every item, build and upload its tables (host arrays are read before
 * the call returns), tune (flags & KB_BATCH_AUTOTUNE; without it the context's
 * variant 1..4 or the default shape) and capture the graph.  Blocks until the
 * uploads and tuning runs are done.  The jobs belong to the batch until
 * kb_batch_free: kb_search on them fails with KB_EINVAL, and they must not be
 * freed before the batch.  The stacks' psi/phi must be complete before each
 * kb_batch_run (the caller orders kb_make_psi_phi before it).  Errors: KB_EINVAL
 * (an item fails kb_search's checks, a job repeated or already in a batch; the
 * message names the item), KB_ENOMEM, KB_ECUDA.  *out: kb_batch_free. */
int kb_batch_create(kb_ctx *ctx, int count, const kb_batch_item *items, int flags, kb_batch **out);

/* Run every search of the batch on `stream` (one graph launch), then record each
 * job's completion so that kb_job_wait / kb_results work per job.  Runs of one
 * batch are serialised by the graph. */
int kb_batch_run(kb_batch *b, void *stream);

/* The batch's groups: *n_groups = their number; up to `capacity` written to out. */
int kb_batch_groups(const kb_batch *b, kb_batch_group *out, int capacity, int *n_groups);

/* Waits for the batch's work, releases it and its jobs (which stay valid). */
void kb_batch_free(kb_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* KB_H */
