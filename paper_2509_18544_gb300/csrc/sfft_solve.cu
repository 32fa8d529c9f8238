// FP64 solve of the normal equations N theta = b (the plain solver): blocked right-looking
// Cholesky N = L L^T with 32 x 32 tiles in ONE cooperative persistent kernel, then forward
// and backward substitution in FP64, and one step of iterative refinement
// (r = b - N theta in FP64, theta += N^{-1} r with an FP32 copy of the factor: the
// correction is ~1e-12 of theta, so its own relative error of ~1e-6 does not matter).
//
// On GB300 the FP64 pipes run at 1/64 of the FP32 rate, so the factorisation of a 732 x 732
// system is bounded by its chain of dependent steps, not by flops; a launch per step spent
// most of its time in launch gaps and cold caches.  Here every CTA of a co-resident grid
// (one per SM) walks the same step sequence: the diagonal tile is factored by CTA 0, the
// panel rows and the trailing tiles are shared by all CTAs, and a grid barrier separates
// the phases.  The barrier's spin has an iteration limit: on expiry it stores
// SFFT_ERR_TIMEOUT in the status word and every CTA returns.  A non-positive pivot stores
// SFFT_ERR_NOT_SPD.  R holds L in its lower and L^T in its upper triangle so both sweeps
// read rows; it is read with ld.global.cg (L2) because other CTAs rewrite it between phases.
#include <math.h>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int NB = 32;
constexpr int CT = 256;

__device__ __forceinline__ double ldg_cg(const double *p) { return __ldcg(p); }

struct SolveArgs {
    const double *N;
    const double *b;
    double *R;
    double *x;      // solution
    double *r;      // residual / refinement rhs
    double *z;      // work vector
    double *scal;   // [0] ||r||^2 after refinement, [1] ||b||^2
    unsigned *bar;  // [0] arrival count, [1] generation
    int *status;
    long long spin_limit;  // barrier wait iterations (~64 ns sleep each) before SFFT_ERR_TIMEOUT
    int n;
    int factor;     // 1: factor N, solve and refine; 0: x += N^{-1} b with the factor in R
    double *dinv;   // [n] reciprocals of the diagonal of L (computed once by the factorisation)
    float *Rf;      // [n][n] FP32 copy of R (L below, L^T above)
    float *dinvf;   // [n] FP32 reciprocals
};

__device__ bool grid_barrier(unsigned *bar, int *status, long long spin_limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (++it > spin_limit) {
                    atomicCAS(status, 0, (int)SFFT_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)status == 0;
}

// factor the diagonal tile kb in place (one CTA)
__device__ void potrf_tile(double *R, double *dinv, float *Rf, float *dinvf, int n, int kb, int *status,
                           double (*a)[NB + 1]) {
    __shared__ int bad;
    __shared__ double inv_s[NB];
    const int r0 = kb * NB, m = min(NB, n - r0);
    for (int e = threadIdx.x; e < NB * NB; e += CT) {
        int rr = e / NB, cc = e % NB;
        if (rr < m && cc < m) a[rr][cc] = ldg_cg(R + (size_t)(r0 + rr) * n + r0 + cc);
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < m; j++) {
        if (threadIdx.x == 0) {
            // one FP64 square root and division per column (FP64 runs at 1/64 of FP32)
            double d = a[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
            } else {
                double sd = sqrt(d);
                a[j][j] = sd;
                inv_s[j] = 1.0 / sd;
            }
        }
        __syncthreads();
        if (bad) break;
        const double inv = inv_s[j];
        if (threadIdx.x > j && threadIdx.x < m) a[threadIdx.x][j] *= inv;
        __syncthreads();
        for (int e = threadIdx.x; e < NB * NB; e += CT) {
            int rr = e / NB, cc = e % NB;
            if (cc > j && rr >= cc && rr < m) a[rr][cc] -= a[rr][j] * a[cc][j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) atomicCAS(status, 0, (int)SFFT_ERR_NOT_SPD);
        return;
    }
    for (int e = threadIdx.x; e < NB * NB; e += CT) {
        int rr = e / NB, cc = e % NB;
        if (rr < m && cc < m) {
            double v = cc <= rr ? a[rr][cc] : a[cc][rr];
            R[(size_t)(r0 + rr) * n + r0 + cc] = v;
            Rf[(size_t)(r0 + rr) * n + r0 + cc] = (float)v;
        }
    }
    if (threadIdx.x < m) {
        dinv[r0 + threadIdx.x] = inv_s[threadIdx.x];
        dinvf[r0 + threadIdx.x] = (float)inv_s[threadIdx.x];
    }
}

// X = A_ib,kb L_kk^{-T}; writes L_ib,kb and its transpose
__device__ void trsm_tile(double *R, float *Rf, const double *dinv, int n, int kb, int ib, double (*Lk)[NB + 1],
                          double (*X)[NB + 1]) {
    const int r0 = kb * NB, m = min(NB, n - r0);
    const int i0 = ib * NB, mi = min(NB, n - i0);
    for (int e = threadIdx.x; e < NB * NB; e += CT) {
        int rr = e / NB, cc = e % NB;
        if (rr < m && cc < m) Lk[rr][cc] = ldg_cg(R + (size_t)(r0 + rr) * n + r0 + cc);
        if (rr < mi && cc < m) X[rr][cc] = ldg_cg(R + (size_t)(i0 + rr) * n + r0 + cc);
    }
    __syncthreads();
    for (int c = 0; c < m; c++) {
        const double inv = ldg_cg(dinv + r0 + c);
        if (threadIdx.x < mi) X[threadIdx.x][c] *= inv;
        __syncthreads();
        for (int e = threadIdx.x; e < NB * NB; e += CT) {
            int rr = e / NB, cc = e % NB;
            if (rr < mi && cc > c && cc < m) X[rr][cc] -= X[rr][c] * Lk[cc][c];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < NB * NB; e += CT) {
        int rr = e / NB, cc = e % NB;
        if (rr < mi && cc < m) {
            R[(size_t)(i0 + rr) * n + r0 + cc] = X[rr][cc];
            R[(size_t)(r0 + cc) * n + i0 + rr] = X[rr][cc];
            Rf[(size_t)(i0 + rr) * n + r0 + cc] = (float)X[rr][cc];
            Rf[(size_t)(r0 + cc) * n + i0 + rr] = (float)X[rr][cc];
        }
    }
    __syncthreads();
}

// A_ib,jb -= L_ib,kb L_jb,kb^T (lower triangle only on the diagonal tile)
__device__ void syrk_tile(double *R, int n, int kb, int ib, int jb, double (*Pi)[NB + 1], double (*Pj)[NB + 1]) {
    const int r0 = kb * NB, m = min(NB, n - r0);
    const int i0 = ib * NB, mi = min(NB, n - i0), j0 = jb * NB, mj = min(NB, n - j0);
    for (int e = threadIdx.x; e < NB * NB; e += CT) {
        int rr = e / NB, cc = e % NB;
        Pi[rr][cc] = (rr < mi && cc < m) ? ldg_cg(R + (size_t)(i0 + rr) * n + r0 + cc) : 0.0;
        Pj[rr][cc] = (rr < mj && cc < m) ? ldg_cg(R + (size_t)(j0 + rr) * n + r0 + cc) : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < m; c++) {
        double bj = Pj[tx][c];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = fma(Pi[ty + 8 * q][c], bj, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int rr = ty + 8 * q;
        if (rr < mi && tx < mj && (ib != jb || tx <= rr)) {
            double *p = R + (size_t)(i0 + rr) * n + j0 + tx;
            *p = ldg_cg(p) - acc[q];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CT) k_cholesky_factor(SolveArgs A, const int *skip) {
    __shared__ double s0[NB][NB + 1];
    __shared__ double s1[NB][NB + 1];
    if (skip && *(volatile const int *)skip == 1) return;  // the fast solver already converged
    const int n = A.n, nblk = (n + NB - 1) / NB;
    for (size_t e = (size_t)blockIdx.x * CT + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * CT)
        A.R[e] = A.N[e];
    if (!grid_barrier(A.bar, A.status, A.spin_limit)) return;
    for (int kb = 0; kb < nblk; kb++) {
        if (blockIdx.x == 0) potrf_tile(A.R, A.dinv, A.Rf, A.dinvf, n, kb, A.status, s0);
        if (!grid_barrier(A.bar, A.status, A.spin_limit)) return;
        const int rest = nblk - kb - 1;
        if (rest == 0) break;
        for (int t = blockIdx.x; t < rest; t += gridDim.x) trsm_tile(A.R, A.Rf, A.dinv, n, kb, kb + 1 + t, s0, s1);
        if (!grid_barrier(A.bar, A.status, A.spin_limit)) return;
        const int ntiles = rest * (rest + 1) / 2;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while ((a + 1) * (a + 2) / 2 <= t) a++;
            while (a * (a + 1) / 2 > t) a--;
            syrk_tile(A.R, n, kb, kb + 1 + a, kb + 1 + (t - a * (a + 1) / 2), s0, s1);
        }
        if (!grid_barrier(A.bar, A.status, A.spin_limit)) return;
    }
}

// Forward then backward substitution with the factor in T precision (R holds L below the
// diagonal and L^T above it), in one CTA: the 32 x 32 diagonal tiles are staged in shared
// memory, the off-diagonal row-dot products run one warp per row.  out = x0 + (L L^T)^{-1} v
// when add, else (L L^T)^{-1} v; v and out are FP64.
template <class T>
__global__ void __launch_bounds__(1024) k_sweeps(const T *__restrict__ R, const T *__restrict__ dinv, int n,
                                                const double *__restrict__ v, double *__restrict__ out, bool add,
                                                const int *__restrict__ status, const int *skip) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *zs = reinterpret_cast<T *>(sm_raw);  // n
    __shared__ T D[NB][NB + 1];
    if (*status || (skip && *(volatile const int *)skip == 1)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) zs[i] = (T)v[i];
    __syncthreads();
    const int nblk = (n + NB - 1) / NB;
    for (int kb = 0; kb < nblk; kb++) {
        const int r0 = kb * NB, m = min(NB, n - r0);
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            int rr = e / NB, cc = e % NB;
            if (rr < m && cc < m) D[rr][cc] = R[(size_t)(r0 + rr) * n + r0 + cc];
        }
        for (int rr = warp; rr < m && kb > 0; rr += nwarp) {
            const T *row = R + (size_t)(r0 + rr) * n;
            T s = 0;
            for (int j = lane; j < r0; j += 32) s += row[j] * zs[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) zs[r0 + rr] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            T zr = lane < m ? zs[r0 + lane] : (T)0;
            const T di = lane < m ? dinv[r0 + lane] : (T)0;
            for (int c = 0; c < m; c++) {
                T zc = __shfl_sync(0xffffffffu, zr, c) * __shfl_sync(0xffffffffu, di, c);
                if (lane == c) zr = zc;
                if (lane > c && lane < m) zr -= D[lane][c] * zc;
            }
            if (lane < m) zs[r0 + lane] = zr;
        }
        __syncthreads();
    }
    for (int kb = nblk - 1; kb >= 0; kb--) {
        const int r0 = kb * NB, m = min(NB, n - r0), r1 = r0 + m;
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            int rr = e / NB, cc = e % NB;
            if (rr < m && cc < m) D[rr][cc] = R[(size_t)(r0 + rr) * n + r0 + cc];
        }
        for (int rr = warp; rr < m && r1 < n; rr += nwarp) {
            const T *row = R + (size_t)(r0 + rr) * n;
            T s = 0;
            for (int j = r1 + lane; j < n; j += 32) s += row[j] * zs[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) zs[r0 + rr] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            T xr = lane < m ? zs[r0 + lane] : (T)0;
            const T di = lane < m ? dinv[r0 + lane] : (T)0;
            for (int c = m - 1; c >= 0; c--) {
                T xc = __shfl_sync(0xffffffffu, xr, c) * __shfl_sync(0xffffffffu, di, c);
                if (lane == c) xr = xc;
                if (lane < c) xr -= D[lane][c] * xc;
            }
            if (lane < m) zs[r0 + lane] = xr;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = (add ? out[i] : 0.0) + (double)zs[i];
}

// r = b - N x (warp per row); with scal, also accumulate ||r||^2 and ||b||^2
__global__ void k_residual(const double *__restrict__ N, const double *__restrict__ b, const double *__restrict__ x,
                           int n, double *__restrict__ r, double *__restrict__ scal, const int *status,
                           const int *skip) {
    if (*status || (skip && *(volatile const int *)skip == 1)) return;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const double *a = N + (size_t)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(a[j], x[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double rv = b[row] - s;
        if (r) r[row] = rv;
        if (scal) {
            atomicAdd(&scal[0], rv * rv);
            atomicAdd(&scal[1], b[row] * b[row]);
        }
    }
}

__global__ void k_zero2(double *scal, const int *skip) {
    if (skip && *(volatile const int *)skip == 1) return;
    scal[0] = 0.0;
    scal[1] = 0.0;
}

int g_coop_grid = 0;

template <class T>
cudaError_t sweeps(const T *R, const T *dinv, int n, const double *v, double *out, bool add, const int *status,
                   const int *skip, cudaStream_t st) {
    size_t smem = sizeof(T) * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(k_sweeps<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    k_sweeps<T><<<1, 1024, smem, st>>>(R, dinv, n, v, out, add, status, skip);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cholesky_solve(const Geometry &g, const double *N, const double *b, double *R, double *x,
                                  double *r, double *z, double *scal, double *dinv, float *Rf, float *dinvf,
                                  unsigned *bar, int *status, bool factor, const int *skip, cudaStream_t st) {
    const int n = g.n;
    cudaError_t e;
    if (!factor) return sweeps<float>(Rf, dinvf, n, b, x, true, status, skip, st);  // x += N^{-1} b
    if (g_coop_grid == 0) {
        int dev = 0, sms = 0, per_sm = 0, coop = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cholesky_factor, CT, 0);
        if (e != cudaSuccess) return e;
        if (!coop || per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        g_coop_grid = sms;  // one CTA per SM: co-resident by construction
    }
    SolveArgs A{N, b, R, x, r, z, scal, bar, status, g.spin_limit, n, 1, dinv, Rf, dinvf};
    void *params[] = {&A, (void *)&skip};
    // As the fallback of PCG (skip != NULL) the factor usually returns at once, but a
    // cooperative launch starts only when all its CTAs can be resident: one CTA per SM would
    // wait for every other stream's kernels to drain.  16 CTAs keep it cheap to schedule;
    // the tile loop runs with any grid, only a real fallback is slower.
    const int grid = skip ? (g_coop_grid < 16 ? g_coop_grid : 16) : g_coop_grid;
    note_launch();
    e = cudaLaunchCooperativeKernel((const void *)k_cholesky_factor, dim3(grid), dim3(CT), params, 0, st);
    if (e != cudaSuccess) return e;
    // FP64 substitution, then one refinement step with the FP32 factor
    if ((e = sweeps<double>(R, dinv, n, b, x, false, status, skip, st)) != cudaSuccess) return e;
    const int rows_per_cta = 8;
    note_launch();
    k_residual<<<(n + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, 0, st>>>(N, b, x, n, r, nullptr, status, skip);
    if ((e = sweeps<float>(Rf, dinvf, n, r, x, true, status, skip, st)) != cudaSuccess) return e;
    note_launch();
    k_zero2<<<1, 1, 0, st>>>(scal, skip);
    note_launch();
    k_residual<<<(n + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, 0, st>>>(N, b, x, n, nullptr, scal, status,
                                                                                    skip);
    return cudaGetLastError();
}

}  // namespace sfft
