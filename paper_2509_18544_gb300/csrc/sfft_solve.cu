// FP64 solve of the normal equations N theta = b: blocked right-looking Cholesky
// N = L L^T (32 x 32 tiles: diagonal factor, panel triangular solve, trailing symmetric
// update, one launch each per block column), forward and backward substitution, and one
// step of iterative refinement (r = b - N theta, theta += N^{-1} r).
//
// The factor array R holds L in its lower triangle and L^T in its upper triangle so both
// substitutions read rows.  A non-positive pivot stores SFFT_ERR_NOT_SPD in the device
// status word; every later kernel of the solve checks the word and returns at once.
#include <math.h>

#include "sfft_internal.cuh"

namespace sfft {
namespace {

constexpr int NB = 32;

__global__ void k_copy(const double *__restrict__ src, double *__restrict__ dst, size_t count) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = src[i];
}

// factor the diagonal block kb in place (1024 threads, one per element)
__global__ void __launch_bounds__(1024) k_potrf(double *R, int n, int kb, int *status) {
    __shared__ double a[NB][NB + 1];
    __shared__ int bad;
    if (*status) return;
    const int r0 = kb * NB, m = min(NB, n - r0);
    const int ty = threadIdx.y, tx = threadIdx.x;
    if (ty < m && tx < m) a[ty][tx] = R[(size_t)(r0 + ty) * n + r0 + tx];
    if (ty == 0 && tx == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < m; j++) {
        if (ty == j && tx == j) {
            double d = a[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
            } else {
                a[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        if (tx == j && ty > j && ty < m) a[ty][j] /= a[j][j];
        __syncthreads();
        if (tx > j && ty >= tx && ty < m) a[ty][tx] -= a[ty][j] * a[tx][j];
        __syncthreads();
    }
    if (bad) {
        if (ty == 0 && tx == 0) atomicCAS(status, 0, (int)SFFT_ERR_NOT_SPD);
        return;
    }
    if (ty < m && tx < m) {
        double v = tx <= ty ? a[ty][tx] : a[tx][ty];  // L below, L^T above
        R[(size_t)(r0 + ty) * n + r0 + tx] = v;
    }
}

// panel: X = A_ib,kb L_kk^{-T} for every row block ib > kb; writes L and its transpose
__global__ void __launch_bounds__(1024) k_trsm(double *R, int n, int kb, const int *status) {
    __shared__ double Lk[NB][NB + 1];
    __shared__ double X[NB][NB + 1];
    if (*status) return;
    const int r0 = kb * NB, m = min(NB, n - r0);
    const int ib = kb + 1 + blockIdx.x;
    const int i0 = ib * NB, mi = min(NB, n - i0);
    const int ty = threadIdx.y, tx = threadIdx.x;
    if (ty < m && tx < m) Lk[ty][tx] = R[(size_t)(r0 + ty) * n + r0 + tx];
    if (ty < mi && tx < m) X[ty][tx] = R[(size_t)(i0 + ty) * n + r0 + tx];
    __syncthreads();
    for (int c = 0; c < m; c++) {
        if (tx == c && ty < mi) X[ty][c] /= Lk[c][c];
        __syncthreads();
        if (tx > c && tx < m && ty < mi) X[ty][tx] -= X[ty][c] * Lk[tx][c];
        __syncthreads();
    }
    if (ty < mi && tx < m) {
        R[(size_t)(i0 + ty) * n + r0 + tx] = X[ty][tx];
        R[(size_t)(r0 + tx) * n + i0 + ty] = X[ty][tx];
    }
}

// trailing update of the lower triangle: A_ib,jb -= L_ib,kb L_jb,kb^T, kb < jb <= ib
__global__ void __launch_bounds__(256) k_syrk(double *R, int n, int kb, const int *status) {
    __shared__ double Pi[NB][NB + 1];
    __shared__ double Pj[NB][NB + 1];
    if (*status) return;
    const int t = blockIdx.x;
    int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((a + 1) * (a + 2) / 2 <= t) a++;
    while (a * (a + 1) / 2 > t) a--;
    const int bcol = t - a * (a + 1) / 2;
    const int ib = kb + 1 + a, jb = kb + 1 + bcol;
    const int r0 = kb * NB, m = min(NB, n - r0);
    const int i0 = ib * NB, mi = min(NB, n - i0), j0 = jb * NB, mj = min(NB, n - j0);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int rr = e / NB, cc = e % NB;
        Pi[rr][cc] = (rr < mi && cc < m) ? R[(size_t)(i0 + rr) * n + r0 + cc] : 0.0;
        Pj[rr][cc] = (rr < mj && cc < m) ? R[(size_t)(j0 + rr) * n + r0 + cc] : 0.0;
    }
    __syncthreads();
    // each thread: 4 outputs (rows ty, ty+8, ty+16, ty+24 of column tx)
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
        if (rr < mi && tx < mj && (ib != jb || tx <= rr)) R[(size_t)(i0 + rr) * n + j0 + tx] -= acc[q];
    }
}

// forward L z = v then backward L^T x = z in one CTA; R holds L (lower) and L^T (upper).
// Each 32 x 32 diagonal block is staged in shared memory before its sequential solve, so
// the 32 dependent steps read shared memory instead of waiting on global loads.
__global__ void __launch_bounds__(1024) k_trsv_both(const double *__restrict__ R, int n, const double *__restrict__ v,
                                                   double *__restrict__ out, const int *status) {
    extern __shared__ double zs[];  // n values, then the staged diagonal block
    __shared__ double D[NB][NB + 1];
    if (*status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) zs[i] = v[i];
    __syncthreads();
    const int nblk = (n + NB - 1) / NB;
    // forward
    for (int kb = 0; kb < nblk; kb++) {
        const int r0 = kb * NB, m = min(NB, n - r0);
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            int rr = e / NB, cc = e % NB;
            if (rr < m && cc < m) D[rr][cc] = R[(size_t)(r0 + rr) * n + r0 + cc];
        }
        if (kb > 0) {
            for (int rr = warp; rr < m; rr += nwarp) {
                const double *row = R + (size_t)(r0 + rr) * n;
                double s = 0.0;
                for (int j = lane; j < r0; j += 32) s = fma(row[j], zs[j], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) zs[r0 + rr] -= s;
            }
        }
        __syncthreads();
        if (warp == 0) {
            double zr = lane < m ? zs[r0 + lane] : 0.0;
            for (int c = 0; c < m; c++) {
                double zc = __shfl_sync(0xffffffffu, zr, c) / D[c][c];
                if (lane == c) zr = zc;
                if (lane > c && lane < m) zr -= D[lane][c] * zc;
            }
            if (lane < m) zs[r0 + lane] = zr;
        }
        __syncthreads();
    }
    // backward with U = L^T (rows of the upper triangle)
    for (int kb = nblk - 1; kb >= 0; kb--) {
        const int r0 = kb * NB, m = min(NB, n - r0), r1 = r0 + m;
        for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
            int rr = e / NB, cc = e % NB;
            if (rr < m && cc < m) D[rr][cc] = R[(size_t)(r0 + rr) * n + r0 + cc];
        }
        if (r1 < n) {
            for (int rr = warp; rr < m; rr += nwarp) {
                const double *row = R + (size_t)(r0 + rr) * n;
                double s = 0.0;
                for (int j = r1 + lane; j < n; j += 32) s = fma(row[j], zs[j], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) zs[r0 + rr] -= s;
            }
        }
        __syncthreads();
        if (warp == 0) {
            double xr = lane < m ? zs[r0 + lane] : 0.0;
            for (int c = m - 1; c >= 0; c--) {
                double xc = __shfl_sync(0xffffffffu, xr, c) / D[c][c];
                if (lane == c) xr = xc;
                if (lane < c) xr -= D[lane][c] * xc;
            }
            if (lane < m) zs[r0 + lane] = xr;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = zs[i];
}

// r = b - N x (warp per row); optional: accumulate ||r||^2 and ||b||^2 into scal[0], scal[1]
__global__ void k_residual(const double *__restrict__ N, const double *__restrict__ b, const double *__restrict__ x,
                           int n, double *__restrict__ r, double *__restrict__ scal, const int *status) {
    if (*status) return;
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

__global__ void k_axpy_final(double *__restrict__ x, const double *__restrict__ d, int n, const int *status) {
    if (*status) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

__global__ void k_zero2(double *scal) {
    scal[0] = 0.0;
    scal[1] = 0.0;
}

}  // namespace

cudaError_t launch_cholesky_solve(const Geometry &g, const double *N, const double *b, double *R, double *x,
                                  double *r, double *z, double *scal, int *status, cudaStream_t st) {
    const int n = g.n;
    const size_t nn = (size_t)n * n;
    note_launch();
    k_copy<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(N, R, nn);
    const int nblk = (n + NB - 1) / NB;
    for (int kb = 0; kb < nblk; kb++) {
        note_launch();
        k_potrf<<<1, dim3(NB, NB), 0, st>>>(R, n, kb, status);
        int rest = nblk - kb - 1;
        if (rest > 0) {
            note_launch();
            k_trsm<<<rest, dim3(NB, NB), 0, st>>>(R, n, kb, status);
            note_launch();
            k_syrk<<<rest * (rest + 1) / 2, 256, 0, st>>>(R, n, kb, status);
        }
    }
    size_t smem = sizeof(double) * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(k_trsv_both, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    k_trsv_both<<<1, 1024, smem, st>>>(R, n, b, x, status);
    // one refinement step
    const int rows_per_cta = 8;
    note_launch();
    k_residual<<<(n + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, 0, st>>>(N, b, x, n, r, nullptr, status);
    note_launch();
    k_trsv_both<<<1, 1024, smem, st>>>(R, n, r, z, status);
    note_launch();
    k_axpy_final<<<(n + 255) / 256, 256, 0, st>>>(x, z, n, status);
    // relative residual after refinement, for the info struct
    note_launch();
    k_zero2<<<1, 1, 0, st>>>(scal);
    note_launch();
    k_residual<<<(n + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, 0, st>>>(N, b, x, n, nullptr, scal, status);
    return cudaGetLastError();
}

}  // namespace sfft
