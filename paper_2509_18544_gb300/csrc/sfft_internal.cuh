// Internal declarations of libsfft: complex arithmetic, the plan object and the kernel
// launchers.  Every launcher queues work on the given stream and returns the launch status.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfft.h"

namespace sfft {

// ------------------------------------------------------------------ complex arithmetic
template <class R>
struct alignas(2 * sizeof(R)) cpx {
    R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__host__ __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// number of monomials of total degree <= d
__host__ __device__ __forceinline__ int npoly(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

// exponents of monomial idx: total degree first, then q ascending
__host__ __device__ __forceinline__ void mono_pq(int idx, int &p, int &q) {
    int d = 0;
    while (idx > d) {
        idx -= d + 1;
        d++;
    }
    q = idx;
    p = d - idx;
}

// ------------------------------------------------------------------ Lanczos-3 window
// Weights of the six taps floor - 2 .. floor + 3 at fractional position f in [0, 1):
// w[j] = L(f - m), m = j - 2, L(t) = sinc(t) sinc(t / 3) = 3 sin(pi t) sin(pi t / 3) / (pi t)^2.
// sin(pi (f - m)) = (-1)^m sin(pi f) serves every tap; sin(pi (f - m) / 3) comes from the
// angle-difference identity on sin/cos(pi f / 3), except for m = 1, where that difference
// cancels as f -> 1, which takes its own sinpi of the (exact) t = f - 1.  f == 0 gives
// exactly (0, 0, 1, 0, 0, 0).  FP32.
__device__ __forceinline__ void lanczos3_taps(float f, float w[6]) {
    if (f == 0.f) {
#pragma unroll
        for (int j = 0; j < 6; j++) w[j] = j == 2 ? 1.f : 0.f;
        return;
    }
    const float s1 = sinpif(f);
    float s3, c3;
    sincospif(f * (1.f / 3.f), &s3, &c3);
    const float h3 = 0.86602540378443864676f;  // sin(pi / 3)
    // sin(pi (f - m) / 3) for m = -2 .. 3
    const float sm[6] = {-0.5f * s3 + h3 * c3, 0.5f * s3 + h3 * c3, s3, sinpif((f - 1.f) * (1.f / 3.f)),
                         -0.5f * s3 - h3 * c3, -s3};
    const float k = 0.30396355092701331433f;  // 3 / pi^2
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const int m = j - 2;
        const float t = f - (float)m;
        const float sg = (m & 1) ? -s1 : s1;
        w[j] = __fdividef(sg * sm[j] * k, t * t);
    }
}

// ------------------------------------------------------------------ geometry of a plan
// The lag correlations are computed per row segment: segment s owns the columns
// [s*U, s*U + U) of every row ("A" side, zero-padded to P) and reads the cyclic window
// [s*U - G, s*U - G + P) ("B" side); G = L - 1 is the largest |lag|, U = P - 2G.
struct Geometry {
    int ny, nx, pitch, L, h, dk, db;
    int nk, nb, nker, n;       // monomials of kernel / background, unknowns
    int P, U, G, nseg, nkf;    // segment FFT length, useful length, halo, segments, half-spectrum bins
    int nimg, nimg_pad;        // spectra per segment row (A then B images), padded to even
    int npair, nent;           // W-W pairs (i <= j), (pair, dy) entries per frequency
    int C, items_per_k, kg;    // y-correlation: dy chunk, work items per frequency, frequencies per CTA
    int kg_ws;                 // frequencies per CTA when only the W x S_m items run (refinement)
    int ytile;                 // y-correlation rows per staged tile
    int ysplit;                // y-correlation row chunks (partial sums per chunk)
    int ychunks_ws;            // row chunks of the refinement (W x S_m) correlation pass
    int refine;                // residual refinement passes after the solve
    int mom_rows, mom_ctas;    // background-moment reduction geometry
    int nmom;                  // moments: npoly(2 db) mask moments + npoly(db) science moments
    int pmax;                  // highest coordinate power tabulated: max(dk, 2 db)
    // launch shape choices (heuristic defaults, or a tuned entry of the process-wide cache)
    int kg_max;                // most y-correlation frequencies per CTA the thread and smem limits allow
    int ycorr_scalar;          // 1: scalar FP32 y-correlation kernel instead of packed FP32x2
    int sub_per_sm;            // subtract / residual CTAs per SM the grid is sized for
    int pcg_cluster;           // PCG cluster size asked for (0: the largest available)
    long long spin_limit;      // iterations of a bounded device-side wait before it gives up
    // y-direction correlation route: 1 = y-block FFTs of the base spectra (K1 writes the
    // nbase x-weighted base images per record), 0 = direct correlation over the rows (K1
    // writes the nimg yh^q-scaled images per record)
    int yfft;
    int nbase, nrec;           // base images per segment row; complex values per spectrum record
    int Py, Uy, nyb;           // y-block FFT length, rows per block, blocks per segment
    int npair_all;             // correlation pairs: npair W-W, then nk (nb + 1) W-(Psi|S)
    int ypg, npg;              // pairs per y-FFT CTA, pair groups
    int y2split, y2split_ws;   // y-FFT CTAs per frequency (main pass, refinement pass)
    int ysets;                 // producer sets of the specialised FP32 y-FFT kernel (1 or 2)
    int subfft;                // difference image by row-segment FFTs (FP32 paths) instead of the direct kernel
};

bool make_geometry(const sfft_desc &d, Geometry &g, char *err, size_t errlen);
// make_geometry, then the cached tuning for this descriptor when there is one
bool plan_geometry(const sfft_desc &d, Geometry &g, char *err, size_t errlen);
// y-correlation row chunks for the current kg: several waves of 2 CTAs on each SM
int default_ysplit(const Geometry &g);

// ------------------------------------------------------------------ plan
struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
    void *spec = nullptr;        // [nseg][ny][nkf][nrec] complex (R)
    double *ypart = nullptr;     // K2 partial sums, 16 bytes per complex value (see the K2 launchers)
    void *resid = nullptr;       // [ny][nx] residual image of the refinement pass (input dtype)
    void *rspec = nullptr;       // [nseg][ny][nkf] complex spectrum of the residual (compact; FP32 path, or y-FFT route)
    double *ysum = nullptr;      // [nkf][nent] complex FP64
    double *lagww = nullptr;     // [npair][2L-1][2L-1]
    double *lagwg = nullptr;     // [nk][nb][L][L]
    double *lagws = nullptr;     // [nk][L][L]
    double *mom_part = nullptr;  // [mom_ctas][nmom]
    double *mom = nullptr;       // [nmom]
    double *N = nullptr;         // [n][n]
    double *b = nullptr;         // [n]
    double *R = nullptr;         // [n][n] Cholesky factor (lower triangle used)
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b2 = nullptr;  // [n] solver vectors
    double *scal = nullptr;      // [16] solver scalars
    double *dinv = nullptr;      // [n] reciprocal diagonal of the Cholesky factor
    float *Rf = nullptr;         // [n][n] FP32 copy of the factor (refinement corrections)
    float *dinvf = nullptr;      // [n] FP32 reciprocal diagonal
    double *dscale = nullptr;    // [n] Jacobi scaling diag(N)^{-1/2} of the fast solver
    float *Lg = nullptr;         // packed FP32 factor tiles of the fast solver
    int *flags = nullptr;        // fast solver: [0] converged, [1] iterations, [2] outcome if not converged
    void *cfold = nullptr;       // subtract: folded kernel coefficients [ny][L][dk+1][L] (R)
    float2 *kspec = nullptr;     // FFT-route subtract: stamp-row spectra [nk][L][128] complex FP32
    int *status = nullptr;       // device status word(s)
    unsigned *bar = nullptr;     // grid-barrier words of the cooperative solver [count, generation]
    void *tw_fft = nullptr;      // [2][P] complex (R): exp(-2 pi i m / P), high part then remainder
    void *xpow = nullptr;        // [pmax+1][nx] (R): xh^p, FP64 powers rounded once
    void *ypow = nullptr;        // [pmax+1][ny] (R): yh^q
    double *tw_x = nullptr;      // [nkf][2G+1] complex FP64: w_k exp(+2 pi i k m / P) / P
    void *tw_y = nullptr;        // [2][Py] complex (R): exp(-2 pi i m / Py), high part then remainder
    void *tw_yi = nullptr;       // [Py] exp(+2 pi i m / Py): FP32 (cos hi, sin hi, cos lo, sin lo) or FP64
};

size_t workspace_bytes(const Geometry &g, int precision, int dtype);

// the warm-start network's output width, batch capacity and current stream
int cnn_n_out(sfft_cnn_t c);
int cnn_max_batch(sfft_cnn_t c);
cudaStream_t cnn_stream(sfft_cnn_t c);

// process-wide count of kernel launches (every launcher calls this before each launch)
void note_launch(int count = 1);
uint64_t launch_count();
// mom[j] = sum over p < nparts of part[p nmom + j], j < nmom (fixed order)
cudaError_t launch_mom_reduce(const double *part, int nparts, int nmom, double *mom, cudaStream_t st);
// largest number of CTAs the FP32 residual kernel can have (sizes its moment partials)
int residual_ctas_max(const Geometry &g);
// residual of the fit on the FP32 paths, in compensated arithmetic (folds the coefficients
// into cfold first); with mom, its background moments go to mom + npoly(2 DB)
cudaError_t launch_residual_comp(const Geometry &g, int dtype, const void *sci, const void *tmpl,
                                 const uint8_t *mask, const double *coeffs, const void *xpow, void *cfold,
                                 void *resid, double *mom_part, double *mom, cudaStream_t st);

enum Stage { ST_SEGFFT = 0, ST_MOMENTS, ST_YCORR, ST_LAGS, ST_ASSEMBLE, ST_SOLVE, ST_SUBTRACT, ST_REFINE, ST_COUNT };

}  // namespace sfft

#include <vector>

struct sfft_plan_s {
    sfft_desc desc;
    sfft::Geometry g;
    sfft::Workspace ws;
    cudaStream_t stream;
    int device;
    char err[512];
    // stage timing: event pairs recorded while profiling, summed on read
    bool profile = false;
    int timed_calls = 0;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[sfft::ST_COUNT];
};

namespace sfft {

// ------------------------------------------------------------------ launchers
// K1: products + row-segment real FFTs -> spec
cudaError_t launch_segment_fft(const Geometry &g, int dtype, int precision, const void *sci,
                               const void *tmpl, const uint8_t *mask, const void *tw_fft, const void *xpow,
                               const void *ypow, void *spec, cudaStream_t st);
// background moments (mask and masked science times monomials) -> mom_part
int moments_ctas(const Geometry &g);  // CTAs (partial sums) of the moments kernel
cudaError_t launch_moments(const Geometry &g, int dtype, int precision, const void *sci,
                           const uint8_t *mask, const void *ypow, double *mom_part, cudaStream_t st);
// K1 for one image (the refinement residual) written into image slot `slot` of spec
cudaError_t launch_segment_fft_single(const Geometry &g, int dtype, int precision, const void *img,
                                      const void *tw_fft, int slot, void *spec, void *rspec, cudaStream_t st);
// K2, y-block FFT route: cross-spectra of the image pairs summed over (segment, block) units,
// one share per CTA -> part [split][nkf][pairs][Py] (16 bytes per value); ws: W_i x R only
size_t yfft_smem_bytes(const Geometry &g, int precision, bool ws);
cudaError_t launch_ycorr_fft(const Geometry &g, int precision, const void *spec, const void *rspec, const void *ypow,
                             const void *tw_y, double *part, bool ws, cudaStream_t st);
// the shares summed and inverted along y at the pairs' lags -> ysum [nkf][nent] (ws: W x S_m entries)
cudaError_t launch_yinv(const Geometry &g, int precision, const double *part, const void *twi, double *ysum, bool ws,
                        cudaStream_t st);
// K2: y-direction correlations at the kernel lags, per segment and frequency -> ypart
// (ws_only: only the W x S_m items)
// (ypow: the FP32 yh^q table, read by the refinement kernel on the y-FFT route)
cudaError_t launch_ycorr(const Geometry &g, int precision, const void *spec, double *ypart, bool ws_only, const void *rspec,
                         const void *ypow, cudaStream_t st);
// K3: segment sum + x-direction inverse DFT at the kernel lags -> lag tables (ws_only: W x S_m only)
// (have_ysum: ysum is already complete -- the y-FFT route -- and only the x-direction
// inverse and the moment reduction run)
cudaError_t launch_lag_tables(const Geometry &g, const double *ypart, double *ysum, const double *tw_x,
                              double *lagww, double *lagwg, double *lagws, const double *mom_part,
                              double *mom, bool ws_only, bool pairs, bool have_ysum, cudaStream_t st);
// refinement right-hand side c = [lagws ; science-moment part of mom]
cudaError_t launch_refine_rhs(const Geometry &g, const double *lagws, const double *mom, double *c,
                              cudaStream_t st);
// K4: normal-matrix and right-hand-side assembly from the lag tables and moments
cudaError_t launch_assemble(const Geometry &g, const double *lagww, const double *lagwg,
                            const double *lagws, const double *mom, double *N, double *b,
                            cudaStream_t st);
// solve N x = b (FP64 Cholesky + one refinement step); writes status on failure.
// factor == false: reuse the factor in R and update x += N^{-1} b instead.
// skip (nullable): device flag; when it reads 1 every kernel of this solve returns at once
// (the fast solver converged and this is its fallback)
cudaError_t launch_cholesky_solve(const Geometry &g, const double *N, const double *b, double *R,
                                  double *x, double *r, double *z, double *scal, double *dinv, float *Rf,
                                  float *dinvf, unsigned *bar, int *status, bool factor, const int *skip,
                                  cudaStream_t st);
// PCG preconditioned by an FP32 Cholesky factor held in one thread-block cluster; flags[0] = 1
// on convergence.  correction: x += M^{-1} b with the stored factor (only if flags[0] == 1).
int pcg_cluster_size(const Geometry &g);  // 0 when the fast solver cannot run this size
size_t pcg_factor_floats(const Geometry &g);
cudaError_t launch_pcg_cluster(const Geometry &g, const double *N, const double *b, const double *x0, double *x,
                               double *r, double *p, double *q, double *z, double *d, float *Lg, double *scal,
                               int *flags, int max_iter, double tol, bool correction, cudaStream_t st);
// difference image (mask == nullptr), or with a mask the residual of the fit on the
// masked frames: S_m - sum a (w T_m)(u - d) - m sum b w
// difference image by row-segment FFTs (FP32 arithmetic); cudaErrorNotSupported where it has
// no kernel (DK > 2, L < 3 or L > 15), and the caller takes launch_subtract
cudaError_t launch_subtract_fft(const Geometry &g, int dtype, const void *sci, const void *tmpl, const double *coeffs,
                                const void *tw_fft, const void *xpow, const void *ypow, float2 *kspec, void *diff,
                                cudaStream_t st);
cudaError_t launch_subtract(const Geometry &g, int dtype, int precision, const void *sci,
                            const void *tmpl, const uint8_t *mask, bool residual, const double *coeffs,
                            const void *xpow, const void *ypow, void *cfold, void *diff, double *mom_part, double *mom, cudaStream_t st);

}  // namespace sfft
