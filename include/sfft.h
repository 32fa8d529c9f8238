/*
 * sfft.h -- C ABI of libsfft, a GB300 (sm_103a) implementation of the SFFT fit and
 * subtraction: the difference-imaging step that fits a spatially varying delta-basis
 * matching kernel plus a polynomial background to a science/template pair and subtracts
 * the convolved template (the SFFT subtraction step, Sec. "Pipeline steps", step 6; the
 * delta basis that follows a spatially varying PSF, Sec. "Statement of need"; the linear
 * system it solves, Sec. "Future development").
 *
 * Problem statement (the paper gives no formulas, so this is the least-squares problem
 * written out; the CPU oracle in oracle/ states the same thing):
 *   frame Ny x Nx, row-major, pixel u = (y, x); xh = 2x/(Nx-1) - 1, yh = 2y/(Ny-1) - 1
 *   (0 on an axis of length 1); monomials w_pq = xh^p yh^q, p+q <= D, ordered by total
 *   degree, then q ascending; mask byte != 0 means "bad pixel" (m = 0), else m = 1;
 *   X_m = m X; cyclic shifts X(u - d) taken modulo the frame.
 *   Unknowns theta = [a_{pq,d}, p+q <= DK, d in [-h,h]^2 (h = (L-1)/2, row-major, dy
 *   outer), pq-major blocks of L^2 lags;  b_rs, r+s <= DB]; n = L^2 nP(DK) + nP(DB),
 *   nP(D) = (D+1)(D+2)/2.
 *   Fit:      theta minimises || S_m - sum a_{pq,d} (w_pq T_m)(u - d) - sum b_rs m w_rs ||^2,
 *             i.e. N theta = b with N, b the normal equations of that design.
 *   Subtract: D(u) = S(u) - sum a_{pq,d} (w_pq T)(u - d) - sum b_rs w_rs(u)  on the
 *             unmasked frames.
 *
 * Conventions for every call:
 *   - Image, mask, coefficient and matrix pointers are caller-owned DEVICE memory on the
 *     plan's device.  Images are row-major with a row pitch of `pitch` elements
 *     (pitch >= nx; 0 means nx); their base pointers must be 16-byte aligned.  Masks are
 *     one byte per pixel with the same pitch.
 *   - The plan owns only its workspace.  All work is issued on the plan's stream and
 *     is stream-ordered; a call returns once its work is queued unless it says it
 *     synchronises.  A plan is not thread-safe; distinct plans on distinct streams are.
 *   - Errors are returned as sfft_status; nothing aborts or traps.  Argument errors are
 *     detected on the host before any work is queued.  Device-side failures (a
 *     non-positive Cholesky pivot, a solver that does not converge) are recorded in a
 *     device status word that sfft_fit reports when it is given an info struct (which
 *     synchronises the stream) and that sfft_sync_status reads otherwise.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *sfft_stream_t;
typedef struct sfft_plan_s *sfft_plan_t;

typedef enum {
    SFFT_OK = 0,
    SFFT_ERR_INVALID_ARG = 1,   /* bad descriptor, pointer, size or alignment */
    SFFT_ERR_CUDA = 2,          /* a CUDA runtime call failed; see sfft_last_error */
    SFFT_ERR_OOM = 3,           /* workspace allocation failed or exceeds workspace_cap */
    SFFT_ERR_NOT_SPD = 4,       /* normal matrix not positive definite (rank-deficient design) */
    SFFT_ERR_NO_CONVERGENCE = 5,/* iterative solver hit max_iter (reported, then fell back) */
    SFFT_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    SFFT_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} sfft_status;

enum { SFFT_F32 = 0, SFFT_F64 = 1 };                              /* input element type */
enum { SFFT_PREC_FP32 = 0, SFFT_PREC_SPLIT = 1, SFFT_PREC_FP64 = 2 }; /* arithmetic */
enum { SFFT_SOLVE_CHOLESKY = 0, SFFT_SOLVE_PCG = 1 };

typedef struct {
    int32_t ny, nx;        /* frame size, ny, nx >= L */
    int32_t pitch;         /* row pitch in elements (>= nx); 0 = nx */
    int32_t L;             /* kernel size, odd, >= 1 */
    int32_t dk;            /* kernel spatial polynomial degree, >= 0 */
    int32_t db;            /* background polynomial degree, >= 0 */
    int32_t dtype;         /* SFFT_F32 or SFFT_F64 (science, template and difference image) */
    int32_t precision;     /* SFFT_PREC_SPLIT: FP32 products and FFTs, cross-spectra summed in
                              FP32 per 64-row tile and folded into split hi/lo pairs, FP64 from
                              the lag tables on, and one refinement pass with a compensated
                              residual (coefficients within ~1e-6 of the FP64 answer);
                              SFFT_PREC_FP32: the same kernels without refinement (faster,
                              ~1e-6 .. 4e-5); SFFT_PREC_FP64: FP64 throughout */
    int32_t solver;        /* SFFT_SOLVE_CHOLESKY (FP64 Cholesky + one refinement step) or
                              SFFT_SOLVE_PCG (PCG in one thread-block cluster: FP32 Cholesky
                              preconditioner of the Jacobi-scaled N, FP64 residuals, warm start
                              from x0; falls back to the FP64 Cholesky on the device when it
                              does not converge or a pivot fails) */
    int32_t max_iter;      /* PCG iteration cap (0 = default) */
    double tol;            /* PCG relative-residual tolerance (0 = default 1e-12) */
    size_t workspace_cap;  /* bytes the plan may allocate; 0 = no cap */
    int32_t seg;           /* row-segment FFT length P (0 = default 256); P >= 2(L-1)+1 */
    int32_t refine;        /* residual refinement passes after the solve: 0 = default (1 for
                              SFFT_PREC_SPLIT, none otherwise), < 0 = none, > 0 = count.
                              A pass forms the residual image of the fit on the masked frames,
                              correlates it with the basis through the same segment spectra,
                              and corrects theta with the existing factorisation. */
    int32_t spin_limit;    /* iteration limit of every bounded device-side wait (the grid
                              barrier of the cooperative FP64 Cholesky): each iteration sleeps
                              ~64 ns, and on expiry the kernel records SFFT_ERR_TIMEOUT in the
                              plan's status word and returns instead of waiting on; 0 = default
                              2^24 (about a second), > 0 = that many iterations */
    int32_t reserved[5];   /* zero */
} sfft_desc;

typedef struct {
    int32_t status;        /* sfft_status of the solve */
    int32_t n;             /* number of unknowns */
    int32_t iterations;    /* solver iterations (refinement steps for Cholesky) */
    int32_t fallback;      /* 1 when PCG fell back to Cholesky */
    double rel_residual;   /* ||b - N theta||_2 / ||b||_2 after the last step */
    double start_residual; /* ||b - N x||_2 / ||b||_2 at PCG's starting point (after the warm
                              start's projection); 1 for Cholesky and for a fallback */
    int32_t pcg_status;    /* SFFT_SOLVE_PCG only: SFFT_OK when PCG met the tolerance,
                              SFFT_ERR_NO_CONVERGENCE when it stopped at max_iter,
                              SFFT_ERR_NOT_SPD when its FP32 preconditioner met a non-positive
                              pivot or a search direction lost positive curvature; in the two
                              error cases the FP64 Cholesky fallback produced the coefficients
                              and `status` is that solve's outcome.  SFFT_OK for Cholesky. */
    int32_t reserved_i;
    double reserved[1];
} sfft_fit_info;

/* Create a plan for one frame geometry and basis.  Validates the descriptor, chooses the
 * segment FFT length, allocates the workspace and uploads FP64-derived twiddle tables.
 * Returns SFFT_ERR_INVALID_ARG (bad descriptor), SFFT_ERR_OOM (allocation or cap),
 * SFFT_ERR_CUDA.  On error *plan is NULL. */
sfft_status sfft_plan(sfft_plan_t *plan, const sfft_desc *desc, sfft_stream_t stream);

/* Release the plan and its workspace (synchronises the plan's stream). NULL is a no-op. */
void sfft_destroy(sfft_plan_t plan);

/* Number of unknowns n = L^2 nP(dk) + nP(db). */
sfft_status sfft_n_unknowns(sfft_plan_t plan, int32_t *n);

/* Workspace bytes a plan for this descriptor allocates (host-only, no allocation). */
sfft_status sfft_workspace_size(const sfft_desc *desc, size_t *bytes);

/* Change the stream later calls are issued on. */
sfft_status sfft_set_stream(sfft_plan_t plan, sfft_stream_t stream);

/* Assemble the normal equations of the fit: N (n x n, row-major, FP64, full symmetric
 * matrix) and b (n, FP64), both device pointers written by the call.  mask may be NULL
 * (no bad pixels).  Order of unknowns as in the header comment. */
sfft_status sfft_normal(sfft_plan_t plan, const void *sci, const void *tmpl, const uint8_t *mask,
                        double *N, double *b);

/* Fit: assemble N, b and solve N theta = b into coeffs (device, n doubles).  x0 (device,
 * n doubles, nullable) is a warm start for SFFT_SOLVE_PCG and ignored by Cholesky.  When
 * info (host) is non-NULL the call synchronises the stream and fills it; the return
 * value then also carries the device-side status (e.g. SFFT_ERR_NOT_SPD). */
sfft_status sfft_fit(sfft_plan_t plan, const void *sci, const void *tmpl, const uint8_t *mask,
                     const double *x0, double *coeffs, sfft_fit_info *info);

/* Difference image diff = S - (fitted kernel applied to the unmasked template) - background,
 * using coeffs (device, n doubles).  diff has the plan's dtype and pitch; it may not alias
 * sci or tmpl. */
sfft_status sfft_subtract(sfft_plan_t plan, const void *sci, const void *tmpl, const double *coeffs,
                          void *diff);

/* Synchronise the plan's stream and return (and clear) the device status word. */
sfft_status sfft_sync_status(sfft_plan_t plan);

/* ---------------------------------------------------------------------------------
 * Batches: the S x T science/template pairs of one object (the pairing of Sec. "Pipeline
 * steps", step 1), each a cutout of its own size.  Pairs are spread over `lanes` streams
 * (longest first onto the least-loaded lane); each lane owns one plan per distinct
 * geometry, so pairs overlap on the GPU.  Pair pointers stay fixed for the batch's life:
 * a run reads the current contents of sci, tmpl, mask and x0 and writes coeffs and diff. */
typedef struct {
    const void *sci, *tmpl;   /* device: first pixel of each cutout (16-byte aligned) */
    const uint8_t *mask;      /* device, nullable */
    const double *x0;         /* device warm start for SFFT_SOLVE_PCG, nullable */
    double *coeffs;           /* device output, n doubles */
    void *diff;               /* device output, ny rows of `pitch` elements */
    int32_t ny, nx;           /* cutout size */
    int32_t pitch;            /* row pitch of the frames the cutouts lie in (elements; 0 = nx) */
    int32_t reserved;
    /* device, nullable: the pair's 18 x 32 x 32 float PSF stamps (the warm-start network's
     * input).  With a network given to sfft_batch_create, every run first evaluates it on
     * the stamps of all pairs that have them and starts their PCG solves from its warm
     * starts (replacing x0). */
    const float *psf_stamps;
    /* Optional pinned host buffers (same pitch as the device ones).  With sci_host set, a run
     * first copies sci_host, tmpl_host and (if both are set) mask_host into sci, tmpl and mask,
     * and after the subtraction copies coeffs into coeffs_host and diff into diff_host (each
     * when set).  The copies run on the pair's lane, so one pair's transfers overlap other
     * pairs' work. */
    const void *sci_host, *tmpl_host;
    const uint8_t *mask_host;
    double *coeffs_host;
    void *diff_host;
} sfft_pair;
typedef struct sfft_batch_s *sfft_batch_t;
enum {
    SFFT_BATCH_GRAPH = 1,     /* capture the whole batch into one CUDA graph; runs replay it */
    SFFT_BATCH_AUTOTUNE = 2   /* autotune every geometry without a cached tuning first */
};
typedef struct sfft_cnn_s *sfft_cnn_t;
/* Build a batch (plans, lanes, and with SFFT_BATCH_GRAPH the graph) and run it once,
 * ordered after the work already queued on `stream`, synchronising before it returns.
 * base supplies L, dk, db, dtype, precision, solver, refine; lanes <= 0 means 4.
 * cnn (nullable): the warm-start network (n_out = L^2 nP(dk)); every run then evaluates it
 * on the psf_stamps of the pairs that carry them, on the creation stream before the pairs
 * fork into the lanes (inside the graph with SFFT_BATCH_GRAPH), and those pairs' solves
 * start from its warm starts.  The network must outlive the batch and may not be used on
 * another stream while a run is in flight. */
sfft_status sfft_batch_create(sfft_batch_t *batch, const sfft_desc *base, const sfft_pair *pairs,
                              int32_t npairs, int32_t lanes, int32_t flags, sfft_cnn_t cnn, sfft_stream_t stream);
/* Queue one run of every pair on the creation stream (one graph launch with
 * SFFT_BATCH_GRAPH). */
sfft_status sfft_batch_run(sfft_batch_t batch);
/* Synchronise and fill infos (host, npairs entries) from the last run; returns the first
 * non-OK pair status (each pair's own is in its info). */
sfft_status sfft_batch_info(sfft_batch_t batch, sfft_fit_info *infos);
void sfft_batch_destroy(sfft_batch_t batch);
/* One-shot: all n_sci x n_tmpl pairs (science-major, pair (i, j) at i*n_tmpl + j), run once
 * and synchronised; cnn (nullable) as for sfft_batch_create; infos (host, nullable)
 * receives each pair's outcome, a non-positive-definite pair is reported there rather than
 * failing the call. */
sfft_status sfft_batch(const sfft_desc *base, int32_t n_sci, int32_t n_tmpl, const sfft_pair *pairs,
                       sfft_cnn_t cnn, sfft_fit_info *infos, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Launch tuning.  Plans take their y-correlation shape and subtract grid density from a
 * process-wide cache keyed by (ny, nx, pitch, L, dk, db, dtype, precision, solver,
 * refine); without an entry built-in heuristics apply.  Zero fields mean "heuristic". */
typedef struct {
    int32_t ycorr_bins;       /* frequencies per y-correlation CTA (1 .. the thread/smem limit) */
    int32_t ycorr_split;      /* y-correlation row chunks (direct) or CTAs per frequency (y-FFT) */
    int32_t ycorr_scalar;     /* 1: scalar FP32 y-correlation kernel, 0: packed FP32x2 */
    int32_t subtract_ctas;    /* subtract / residual CTAs per SM the grid is sized for (1 .. 4) */
    int32_t pcg_cluster;      /* CTAs in the PCG solver's cluster: 8 or 16 (0 = the largest the
                                 device allows); a smaller cluster is easier to place among the
                                 other lanes of a batch */
    int32_t ycorr_direct;     /* 0: y-block FFT route (K1 writes the x-weighted base spectra; the
                                 y correlation takes 128-point DFTs of 128-row blocks and inverts
                                 the summed cross-spectra at the lags; ycorr_split = CTAs per
                                 frequency); 1: direct correlation over the rows (K1 writes every
                                 image's spectrum; ycorr_bins, ycorr_split, ycorr_scalar apply) */
    int32_t ycorr_sets;       /* y-block FFT route, DK, DB <= 2: producer warp sets transforming
                                 row blocks concurrently, 1 or 2 (0 = the default, 2) */
    int32_t subtract_fft;     /* FP32 paths, DK <= 2, 3 <= L <= 15, DB <= 4: 1 = difference image by
                                 256-point row-segment FFTs, 0 = the direct kernel (default) */
} sfft_tuning;
/* The cached entry for desc (zeros and *cached = 0 when there is none). */
sfft_status sfft_tuning_get(const sfft_desc *desc, sfft_tuning *t, int32_t *cached);
/* Validate t against desc's limits and store it (SFFT_ERR_INVALID_ARG when out of range). */
sfft_status sfft_tuning_set(const sfft_desc *desc, const sfft_tuning *t);
/* Time candidate shapes on the given pair (device images; coordinate descent over the
 * y-correlation kernel variant and bins, then its row split, then the subtract density;
 * best of `trials` fit+subtract runs each, CUDA events), store the fastest and return it
 * with its time in ms (best, best_ms: host, nullable).  Synchronises. */
sfft_status sfft_autotune(const sfft_desc *desc, const void *sci, const void *tmpl, const uint8_t *mask,
                          int32_t trials, sfft_tuning *best, double *best_ms);
/* Write / read the whole cache as text, one entry per line. */
sfft_status sfft_tuning_save(const char *path);
sfft_status sfft_tuning_load(const char *path);

/* Difference image exactly like sfft_subtract, but without a plan and without allocating:
 * no cudaMalloc, no cudaFree, no library routine that allocates.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device memory at
 * the point where they need the difference image -- for example code whose device memory
 * is owned by another allocator (a framework's caching allocator or a fixed-size arena that
 * must not be bypassed) or a latency-critical path that cannot afford the implicit device
 * synchronisation cudaMalloc and cudaFree may perform.
 *
 * desc gives the frame geometry, basis, dtype and precision (solver fields are ignored);
 * sci, tmpl, coeffs (n doubles) and diff are device pointers as for sfft_subtract, with
 * pitch = desc->pitch (0 = nx), queued on `stream`.  The scratch -- the coordinate-power
 * table and the folded kernel coefficients, (max(dk,db)+1) nx + ny (L^2 (dk+1) + db + 1)
 * values of 4 bytes (8 for SFFT_PREC_FP64) -- lives in one fixed 16 MiB device array.  The
 * array is created on a device when the library's kernels are first loaded there (with
 * CUDA's lazy module loading that can be during the first call of this entry point, or of
 * any other libsfft call) and stays until the process exits; a frame that needs more is
 * rejected with SFFT_ERR_INVALID_ARG (message in sfft_last_error(NULL)).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress, once per
 * device, with the device current) and keeps it; make that first call (a warm-up call is
 * enough) before any stream capture or latency-critical use.  The kept address belongs to
 * the device's primary context: after cudaDeviceReset it is stale, so do not use this
 * entry point on a device that this process has reset.  All calls share the array and
 * each call overwrites everything it reads, so nothing carries over from the previous
 * call, but calls that overlap on the GPU (different streams, or different host threads
 * on one device) race on it and must be serialised. */
sfft_status sfft_subtract_noalloc(const sfft_desc *desc, const void *sci, const void *tmpl,
                                  const double *coeffs, void *diff, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Cross-convolution (Sec. "Pipeline steps", step 5: before the subtraction the science
 * image is convolved with the template's PSF and the template with the science image's,
 * so that both carry the same PSF).
 *   sci_out(u)  = sum_d psf_tmpl(d) sci((u - d) mod N),
 *   tmpl_out(u) = sum_d psf_sci(d)  tmpl((u - d) mod N),
 * d = (a - r, b - r) for stamp element [a][b] of the K x K row-major float32 stamps
 * (K = 2r + 1 odd, 1 <= K <= 31, centred on the middle element), cyclic on the ny x nx
 * frame.  Images and outputs are device arrays of `dtype` (SFFT_F32 or SFFT_F64) with a row
 * pitch of `pitch` elements (0 = nx); the arithmetic is FP32 (direct sums for K < 9, 256-point
 * row-segment FFTs for K >= 9).  Either half is skipped when
 * its image, stamp or output is NULL (both NULL: SFFT_ERR_INVALID_ARG); an output may not
 * alias an input.  Queued on `stream`; no allocation. */
sfft_status sfft_cross_convolve(int32_t ny, int32_t nx, int32_t pitch, int32_t dtype, int32_t K, const void *sci,
                                const void *tmpl, const float *psf_sci, const float *psf_tmpl, void *sci_out,
                                void *tmpl_out, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Alignment and resampling (Sec. "Pipeline steps", step 4: the template image, its
 * detection mask and its PSF are aligned to the science frame on the GPU; Sec. "GPU
 * acceleration and performance" names alignment and resampling as where much of the
 * porting effort went).  The paper fixes neither a coordinate model nor an interpolation
 * kernel; the library's definitions:
 *   coordinates   science pixel (x, y) (column, row) reads template position (u, v),
 *                 u = sum_j cu[j] (x - x_ref)^p_j (y - y_ref)^q_j, v likewise with cv, over
 *                 the first (degree + 1)(degree + 2)/2 monomials of (0,0), (1,0), (0,1),
 *                 (2,0), (1,1), (0,2), (3,0), (2,1), (1,2), (0,3) (p = x power), degree 1..3:
 *                 the affine part of two WCS solutions plus a low-order distortion between
 *                 them, fitted by the caller;
 *   interpolation Lanczos-3 (taps floor(u) - 2 .. floor(u) + 3, window sinc(t) sinc(t/3),
 *                 exactly 1 at t = 0 and 0 at the other integers) or bilinear, separable,
 *                 normalised by the sum of all tap weights;
 *   bad taps      a tap with non-zero weight that falls outside the template or on a masked
 *                 pixel (mask byte != 0) adds no value and its pixel is not read; out_mask = 1
 *                 where more than 1 % of the taps' |weight| is bad.  With
 *                 SFFT_RESAMPLE_ZERO_OUTSIDE outside taps are zeros and are not bad (stamps);
 *   flux          SFFT_RESAMPLE_FLUX multiplies by |det d(u,v)/d(x,y)| (values are fluxes
 *                 per pixel and the pixel area changes).
 * Coordinates are evaluated in FP64 at the corner of each 32 x 32 output tile and by an FP32
 * Taylor expansion inside it (error a few 1e-6 pixel); weights and sums are FP32. */
typedef struct {
    int32_t degree;            /* 1 .. 3 */
    int32_t reserved;          /* 0 */
    double x_ref, y_ref;       /* origin of the polynomials, science pixels */
    double cu[10], cv[10];     /* coefficients in the monomial order above; the tail past the
                                  degree's count is ignored */
} sfft_warp;
enum { SFFT_LANCZOS3 = 0, SFFT_BILINEAR = 1 };
enum { SFFT_RESAMPLE_FLUX = 1, SFFT_RESAMPLE_ZERO_OUTSIDE = 2 };
/* Resample `in` (in_ny x in_nx, row pitch in_pitch elements, 0 = in_nx; dtype SFFT_F32 or
 * SFFT_F64; device) onto the out_ny x out_nx science grid `out` (same dtype, pitch out_pitch,
 * 0 = out_nx; device).  in_mask / out_mask: device bytes with the image's pitch, each
 * nullable.  warp: host struct, copied.  Queued on `stream`; no allocation.
 * SFFT_ERR_INVALID_ARG on a bad size, degree, method, flag or an output aliasing an input. */
sfft_status sfft_resample(const sfft_warp *warp, int32_t method, int32_t flags, int32_t in_ny, int32_t in_nx,
                          int32_t in_pitch, int32_t dtype, const void *in, const uint8_t *in_mask, int32_t out_ny,
                          int32_t out_nx, int32_t out_pitch, void *out, uint8_t *out_mask, sfft_stream_t stream);
/* The template PSF aligned to the science grid at science position (x, y): with J the warp's
 * Jacobian at (x, y) (host, FP64), output stamp offset d reads template stamp offset J d;
 * Lanczos-3, zeros outside the stamp, flux-conserving (|det J|).  psf_in, psf_out: device
 * K x K float32 stamps centred on the middle element, K odd, 1 <= K <= 63, not aliased. */
sfft_status sfft_align_psf(const sfft_warp *warp, double x, double y, int32_t K, const float *psf_in,
                           float *psf_out, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Decorrelation kernel (Sec. "Pipeline steps", step 7: fitted, then applied to the
 * difference image, the science PSF and the cross-convolved science image).  The paper
 * cites the kernel without a formula; the library's definition: the fit matches
 * S' = S (x) P_T against T' = T (x) P_S, so white pixel noise sigma_S, sigma_T leaves
 * D = S' - K (x) T' with the noise spectrum
 *     den(k) = sigma_S^2 |P_T(k)|^2 + sigma_T^2 |K(k)|^2 |P_S(k)|^2,
 * and the kernel whitens it at unit gain for a point source's flux:
 *     Phi(k) = sqrt(num / max(den(k), 1e-8 num)),   num = sigma_S^2 + K(0)^2 sigma_T^2,
 * on the M x M cyclic grid (every stamp centred on it, offset d at index d mod M);
 * phi = IDFT(Phi) and the decorrelated science PSF IDFT(P_S P_T Phi) are written as centred
 * M x M float32 stamps.  K(d) is the fitted matching kernel at science pixel (x, y):
 * K(d) = sum_pq a_{pq,d} xh^p yh^q from the first L^2 nP(dk) entries of `coeffs` (the fit's
 * theta, device FP64; xh, yh normalised on the ny x nx frame).  psf_sci, psf_tmpl: device
 * K x K float32 stamps (the cross-convolution's); M odd with max(K, L) <= M <= 31 so that
 * sfft_cross_convolve can apply phi (to D and to the cross-convolved science image, one call);
 * sigma_sci > 0, sigma_tmpl >= 0.  DFTs and Phi in FP64.  psf_out nullable.  One CTA,
 * queued on `stream`; no allocation. */
sfft_status sfft_decorrelation_kernel(int32_t ny, int32_t nx, int32_t L, int32_t dk, const double *coeffs,
                                      double x, double y, int32_t K, const float *psf_sci,
                                      const float *psf_tmpl, double sigma_sci, double sigma_tmpl, int32_t M,
                                      float *phi, float *psf_out, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Forced PSF photometry (Sec. "Pipeline steps", step 9: the PSF fitted to the decorrelated
 * difference image at the transient's coordinates; step 8 fits the same PSF to field stars).
 * One job = one image and one position; a launch takes any number of jobs (all pairs of a
 * batch, or many stars of one image).  Definition: the source at (x, y) sits on pixel
 * (X, Y) = (floor(x + 0.5), floor(y + 0.5)) with offset (fx, fy) = (x - X, y - Y); the model
 * P(a, b) is the K x K stamp moved by (fx, fy) (Lanczos-3 as in sfft_resample, zeros outside
 * the stamp), placed on the footprint (Y + a, X + b), |a|, |b| <= (K - 1)/2.  Footprint
 * pixels inside the frame, unmasked and with weight > 0 enter
 *     minimise sum w (D - f P - b)^2    (b = 0 unless SFFT_PHOT_BACKGROUND),
 * solved from the 1 x 1 or 2 x 2 normal equations in FP64. */
typedef struct {
    const void *image;     /* device ny x pitch, dtype */
    const float *weight;   /* device inverse variances with the image's pitch; NULL = all 1 */
    const uint8_t *mask;   /* device bytes with the image's pitch, non-zero = excluded; nullable */
    const float *psf;      /* device K x K float32 stamp centred on its middle element */
    double x, y;           /* source position, pixels (column, row) */
    int32_t ny, nx, pitch, dtype;  /* pitch in elements (0 = nx); SFFT_F32 or SFFT_F64 */
} sfft_phot_job;
enum { SFFT_PHOT_BACKGROUND = 1 };
/* jobs: device array of njobs entries (caller-owned, read by the kernel).  results: device,
 * 8 doubles per job: flux, formal flux error sqrt([(A^T W A)^-1]_ff), background (0 without
 * the flag), chi2 = sum w r^2, pixels used, status (0 = solved, 1 = no usable pixel or a
 * singular system: the other fields 0), 0, 0.  K odd, 1 <= K <= 63.  Queued on `stream`;
 * no allocation; per-job problems are reported in `status`, not as a call error. */
sfft_status sfft_forced_photometry(int32_t njobs, const sfft_phot_job *jobs, int32_t K, int32_t flags,
                                   double *results, sfft_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Warm-start network (the learned warm start of the PCG solve).  A small CNN maps the
 * point-spread functions of a pair -- 32 x 32 stamps of unit mean at the centres of a
 * 3 x 3 grid over the frame, 18 channels ordered (cell row-major, then science, template)
 * -- to the n_out = L^2 nP(DK) kernel coefficients of the fit in the unknowns' order.  It
 * is trained on coefficients that sfft_fit produces.  The paper has no network; it
 * stands in for the prior knowledge of how a kernel follows the two PSFs.
 *   layers: 4 x [3x3 conv, stride 2, zero pad 1, 32 ch, ReLU] (32 -> 2 px), flatten
 *           (channel, row, column), linear 128 -> n_out;
 *   parameters: one float vector, conv1 W[32][18][3][3], b[32], conv2 W[32][32][3][3], b,
 *           conv3, conv4 likewise, linear W[n_out][128], b[n_out];
 *   loss: mean squared error; optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * All pointers are device memory except where marked host; calls are queued on the
 * network's stream.  Stamps are [batch][18][32][32] float, targets and outputs
 * [batch][n_out] float.  A network is not thread-safe. */
/* Allocate a network (parameters, Adam moments, activations for up to max_batch samples),
 * zero-initialised; SFFT_ERR_OOM if the allocation fails. */
sfft_status sfft_cnn_create(sfft_cnn_t *cnn, int32_t n_out, int32_t max_batch, sfft_stream_t stream);
void sfft_cnn_destroy(sfft_cnn_t cnn);
sfft_status sfft_cnn_param_count(sfft_cnn_t cnn, int64_t *count /* host */);
/* Change the stream later calls are queued on. */
sfft_status sfft_cnn_set_stream(sfft_cnn_t cnn, sfft_stream_t stream);
/* Copy params (host or device, param_count floats) in; resets the Adam moments and step.
 * Synchronises the stream. */
sfft_status sfft_cnn_set_params(sfft_cnn_t cnn, const float *params);
/* Copy the parameters out (host or device); synchronises the stream. */
sfft_status sfft_cnn_get_params(sfft_cnn_t cnn, float *params);
sfft_status sfft_cnn_forward(sfft_cnn_t cnn, const float *stamps, int32_t batch, float *out);
/* Loss and gradients without an update: grad (param_count floats), grad_in (the stamps'
 * gradient, nullable), loss (1 float, nullable). */
sfft_status sfft_cnn_gradients(sfft_cnn_t cnn, const float *stamps, const float *targets, int32_t batch,
                               float *grad, float *grad_in, float *loss);
/* One Adam step on one batch; loss (1 float, nullable) receives the batch's loss before the update. */
sfft_status sfft_cnn_train_step(sfft_cnn_t cnn, const float *stamps, const float *targets, int32_t batch,
                                float lr, float *loss);
/* `epochs` passes over n samples in minibatches of `batch`, reshuffled every epoch by a
 * host SplitMix64 stream seeded with `seed` (the ragged remainder is skipped).
 * epoch_loss (host, epochs floats, nullable) receives each epoch's mean minibatch loss.
 * Synchronises the stream once per epoch. */
sfft_status sfft_cnn_train(sfft_cnn_t cnn, const float *stamps, const float *targets, int32_t n, int32_t batch,
                           int32_t epochs, float lr, uint64_t seed, float *epoch_loss);
/* Warm starts for sfft_fit: x0[b n_stride + j] = output j of sample b (j < n_out), 0 for
 * the remaining n_stride - n_out unknowns (the background). */
sfft_status sfft_cnn_warm_start(sfft_cnn_t cnn, const float *stamps, int32_t batch, int32_t n_stride, double *x0);
/* Parameters to and from a file (a trained network kept between runs): an 8-byte tag
 * "SFFTCNN1", int32 n_out, int32 0, int64 param_count, then param_count floats, all in the
 * host's byte order (little-endian on x86-64 and AArch64).  Load reads the whole file, checks
 * tag, n_out and count against this network and returns SFFT_ERR_INVALID_ARG on a mismatch,
 * a short or unreadable file; on success it replaces the parameters and resets the Adam
 * state like sfft_cnn_set_params.  Both synchronise the network's stream. */
sfft_status sfft_cnn_save(sfft_cnn_t cnn, const char *path);
sfft_status sfft_cnn_load(sfft_cnn_t cnn, const char *path);
const char *sfft_cnn_last_error(sfft_cnn_t cnn);

/* Stage timing (instrumentation; the paper profiles its pipeline stage by stage, Sec. "GPU
 * acceleration and performance").  With enable != 0 every later call records CUDA events
 * around its stages on the plan's stream.  sfft_stage_times synchronises the stream, adds
 * the elapsed milliseconds of all calls since the previous read into ms[0..SFFT_NSTAGES-1]
 * (host array, caller-owned; order: segment FFT, background moments, y-correlation, lag
 * tables, assembly, solve, subtract, refinement), sets *calls to the number of timed calls,
 * and resets the accumulators. */
enum { SFFT_NSTAGES = 8 };
sfft_status sfft_profile(sfft_plan_t plan, int32_t enable);
sfft_status sfft_stage_times(sfft_plan_t plan, double *ms, int32_t *calls);

/* Process-wide number of kernel launches libsfft has issued (host counter). */
sfft_status sfft_launch_count(uint64_t *count);

const char *sfft_status_string(sfft_status s);
/* Last error message recorded on this plan (or the process-wide one for plan == NULL). */
const char *sfft_last_error(sfft_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H */
