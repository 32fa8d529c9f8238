// PCG solve of the normal equations N theta = b, preconditioned by an FP32 Cholesky factor
// held in the distributed shared memory of one thread-block cluster.
//
// GB300 runs FP64 at 2 FMA / clock / SM (1/64 of FP32), so an FP64 factorisation is bound by
// its chain of dependent steps.  Here one cluster of CL CTAs (16 where the device allows a
// non-portable cluster of that size, else 8) keeps the Jacobi-scaled matrix
//   A = D N D,  D = diag(N)^{-1/2}
// as FP32 lower-triangular 32 x 32 tiles spread round-robin over the CTAs' shared memory,
// factors it right-looking with hardware cluster barriers (A = L L^T), and then runs
// preconditioned conjugate gradients on N theta = b in FP64 with M^{-1} = D (L L^T)^{-1} D.
// The residuals and matrix-vector products are FP64 (N is read from global memory), so the
// solution reaches FP64 accuracy; the FP32 factor only has to be a good preconditioner
// (cond(A) * n * 2^-24 << 1), which makes the iteration converge in a few steps.
//
// Outcome flags (device): flag[0] = 1 when PCG met the tolerance; otherwise 0, and the
// caller's stream-ordered fallback (the FP64 Cholesky) runs.  A non-positive FP32 pivot or a
// non-finite value also leaves flag[0] = 0.  A warm start x0 (nullable) is replaced by the
// Galerkin projection of the solution onto span{x0, background unit vectors}: the starting
// point alpha x0 + sum_r beta_r e_r minimising the N-norm error, from a (1 + nB) system
// (a warm start that predicts the kernel coefficients leaves the background to this
// projection).  Mode 1 reuses the factor stored in global memory by a
// mode-0 call and applies one preconditioned correction x += M^{-1} c (refinement passes).
#include <cooperative_groups.h>
#include <math.h>

#include "sfft_internal.cuh"

namespace cg = cooperative_groups;

namespace sfft {
namespace {

constexpr int TB = 32;          // tile size
constexpr int TS = 33;          // tile row stride (column 32 holds the reciprocal diagonal)
constexpr int TT = TB * TS;     // floats per tile
constexpr int CTH = 256;        // threads per CTA

struct FastArgs {
    const double *N;
    const double *b;   // right-hand side (mode 1: the correction right-hand side c)
    const double *x0;  // warm start (nullable)
    double *x;         // solution (mode 1: updated in place)
    double *r, *p, *q, *z, *d;  // [n] FP64 work vectors, d = diag(N)^{-1/2}
    float *Lg;         // packed FP32 factor tiles in global memory [ntiles][TT]
    double *scal;      // [0] final ||r||^2, [1] ||b||^2, [2] ||r||^2 at the starting point
    int *flags;        // [0] converged, [1] iterations, [2] outcome when not converged (sfft_status)
    int n, nblk, ntiles;
    int nker, nb;      // kernel and background unknowns (n = nker + nb)
    int max_iter;
    double tol;
    int mode;
};

__device__ __forceinline__ void tile_ij(int t, int &i, int &j) {
    int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= t) a++;
    while (a * (a + 1) / 2 > t) a--;
    i = a;
    j = t - a * (a + 1) / 2;
}
__device__ __forceinline__ int tile_id(int i, int j) { return i * (i + 1) / 2 + j; }

constexpr int kGalMax = 11;  // warm-start projection for up to 10 background terms (DB <= 3)

// Solves the m x m system held as the augmented m x (m + 1) matrix a (overwritten) by
// Gaussian elimination with partial pivoting; a column without a usable pivot (relative
// size < 1e-13) gets the value 0.  One thread.
__device__ void solve_small(double *a, int m, double *x) {
    const int w = m + 1;
    int prow[kGalMax];
    double amax = 0.0;
    for (int e = 0; e < m * w; e++) amax = fmax(amax, fabs(a[e]));
    int r = 0;
    for (int c = 0; c < m; c++) {
        int best = -1;
        double bv = 1e-13 * amax;
        for (int i = r; i < m; i++)
            if (fabs(a[i * w + c]) > bv) bv = fabs(a[i * w + c]), best = i;
        if (best < 0 || !isfinite(bv)) {
            prow[c] = -1;
            continue;
        }
        if (best != r)
            for (int j = 0; j < w; j++) {
                double t = a[r * w + j];
                a[r * w + j] = a[best * w + j];
                a[best * w + j] = t;
            }
        for (int i = r + 1; i < m; i++) {
            const double f = a[i * w + c] / a[r * w + c];
            for (int j = c; j < w; j++) a[i * w + j] -= f * a[r * w + j];
        }
        prow[c] = r++;
    }
    for (int c = m - 1; c >= 0; c--) {
        if (prow[c] < 0) {
            x[c] = 0.0;
            continue;
        }
        const int i = prow[c];
        double s = a[i * w + m];
        for (int j = c + 1; j < m; j++) s -= a[i * w + j] * x[j];
        x[c] = s / a[i * w + c];
    }
}

// copy a 32 x 32 tile (stride TS) from src (possibly another CTA's shared memory) to dst
__device__ __forceinline__ void copy_tile(float *dst, const float *src) {
    for (int e = threadIdx.x; e < TT; e += CTH) dst[e] = src[e];
}

// sum of one double per CTA over the cluster (every CTA gets the same value, same order)
__device__ double cluster_sum(cg::cluster_group &cl, double *slot, double v) {
    __shared__ double red[CTH / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < CTH / 32; k++) s += red[k];
        *slot = s;
    }
    cl.sync();
    double tot = 0.0;
    for (unsigned rk = 0; rk < cl.num_blocks(); rk++) tot += *cl.map_shared_rank(slot, rk);
    cl.sync();  // slots may be reused after everybody has read them
    return tot;
}

__global__ void __launch_bounds__(CTH) k_pcg_cluster(FastArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
    extern __shared__ __align__(16) float smem[];
    const int ntl = (A.ntiles + CL - 1) / CL;  // tiles per CTA (upper bound)
    float *tiles = smem;                        // [ntl][TT]
    float *sA = tiles + (size_t)ntl * TT;       // scratch tiles
    float *sB = sA + TT;
    float *sI = sB + TT;                        // inverse of the diagonal factor tile (owner only)
    float *v = sI + TT;                         // [nblk*TB] sweep vector (each CTA holds a copy)
    __shared__ double slot;
    __shared__ int bad;
    // correction mode runs only when a converged mode-0 call left a valid factor
    if (A.mode == 1 && *(volatile int *)A.flags != 1) return;
    const int n = A.n, nblk = A.nblk, npad = nblk * TB;
    const int tid = threadIdx.x;
    auto owner = [&](int t) { return t % CL; };
    auto local = [&](int t) { return tiles + (size_t)(t / CL) * TT; };
    auto remote = [&](int t) { return cl.map_shared_rank(tiles, owner(t)) + (size_t)(t / CL) * TT; };

    if (tid == 0) bad = 0;
    // Jacobi scaling d_i = 1 / sqrt(N_ii), once per row (FP64 square roots and divides run on
    // the narrow FP64 pipe), visible to the whole cluster before the tiles are loaded
    if (A.mode == 0) {
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) A.d[i] = 1.0 / sqrt(A.N[(size_t)i * n + i]);
        cl.sync();
    }
    // ---------------------------------------------------------------- load the tiles
    for (int t = rank; t < A.ntiles; t += CL) {
        int bi, bj;
        tile_ij(t, bi, bj);
        float *T = local(t);
        for (int e = tid; e < TB * TB; e += CTH) {
            int rr = e / TB, cc = e % TB;
            int gi = bi * TB + rr, gj = bj * TB + cc;
            float val;
            if (A.mode == 1) {
                val = A.Lg[(size_t)t * TT + rr * TS + cc];
            } else if (gi < n && gj < n) {
                val = (float)(A.N[(size_t)gi * n + gj] * __ldcg(A.d + gi) * __ldcg(A.d + gj));
            } else {
                val = (gi == gj) ? 1.0f : 0.0f;  // identity padding past n
            }
            T[rr * TS + cc] = val;
        }
        if (A.mode == 1 && bi == bj)
            for (int rr = tid; rr < TB; rr += CTH) T[rr * TS + TB] = A.Lg[(size_t)t * TT + rr * TS + TB];
    }
    cl.sync();

    // ---------------------------------------------------------------- factorise (mode 0)
    if (A.mode == 0) {
        for (int kb = 0; kb < nblk; kb++) {
            const int td = tile_id(kb, kb);
            if (owner(td) == rank) {
                float *a = local(td);
                for (int j = 0; j < TB; j++) {
                    if (tid == 0) {
                        float dj = a[j * TS + j];
                        if (!(dj > 0.0f) || !isfinite(dj)) {
                            bad = 1;
                            dj = 1.0f;
                        }
                        float sd = sqrtf(dj);
                        a[j * TS + j] = sd;
                        a[j * TS + TB] = 1.0f / sd;  // reciprocal diagonal in the pad column
                    }
                    __syncthreads();
                    const float inv = a[j * TS + TB];
                    if (tid > j && tid < TB) a[tid * TS + j] *= inv;
                    __syncthreads();
                    for (int e = tid; e < TB * TB; e += CTH) {
                        int rr = e / TB, cc = e % TB;
                        if (cc > j && rr >= cc) a[rr * TS + cc] -= a[rr * TS + j] * a[cc * TS + j];
                    }
                    __syncthreads();
                }
                // inverse of the lower-triangular tile, one column per thread (tid < 32)
                if (tid < TB) {
                    const int c = tid;
                    for (int rr = 0; rr < TB; rr++) {
                        float s = (rr == c) ? 1.0f : 0.0f;
                        for (int k = c; k < rr; k++) s -= a[rr * TS + k] * sI[k * TS + c];
                        sI[rr * TS + c] = rr >= c ? s * a[rr * TS + TB] : 0.0f;
                    }
                }
            }
            cl.sync();
            if (kb + 1 == nblk) break;
            // panel: L_ik = A_ik L_kk^{-T} = A_ik (L_kk^{-1})^T for the tiles this CTA owns
            bool have_inv = false;
            for (int ib = kb + 1; ib < nblk; ib++) {
                const int t = tile_id(ib, kb);
                if (owner(t) != rank) continue;
                if (!have_inv) {
                    if (owner(td) != rank) copy_tile(sB, cl.map_shared_rank(sI, owner(td)));
                    else copy_tile(sB, sI);
                    have_inv = true;
                    __syncthreads();
                }
                float *X = local(t);
                copy_tile(sA, X);
                __syncthreads();
                for (int e = tid; e < TB * TB; e += CTH) {
                    int rr = e / TB, cc = e % TB;
                    float s = 0.0f;
                    for (int k = 0; k <= cc; k++) s += sA[rr * TS + k] * sB[cc * TS + k];
                    X[rr * TS + cc] = s;
                }
                __syncthreads();
            }
            cl.sync();
            // trailing update A_ij -= L_ik L_jk^T, kb < j <= i
            for (int ib = kb + 1; ib < nblk; ib++)
                for (int jb = kb + 1; jb <= ib; jb++) {
                    const int t = tile_id(ib, jb);
                    if (owner(t) != rank) continue;
                    const int ti = tile_id(ib, kb), tj = tile_id(jb, kb);
                    copy_tile(sA, owner(ti) == rank ? local(ti) : remote(ti));
                    copy_tile(sB, owner(tj) == rank ? local(tj) : remote(tj));
                    __syncthreads();
                    float *Ct = local(t);
                    for (int e = tid; e < TB * TB; e += CTH) {
                        int rr = e / TB, cc = e % TB;
                        if (ib == jb && cc > rr) continue;
                        float s = 0.0f;
#pragma unroll 8
                        for (int k = 0; k < TB; k++) s += sA[rr * TS + k] * sB[cc * TS + k];
                        Ct[rr * TS + cc] -= s;
                    }
                    __syncthreads();
                }
            cl.sync();
        }
        // keep the factor for later correction solves, and decide on the pivots
        for (int t = rank; t < A.ntiles; t += CL) {
            const float *T = local(t);
            for (int e = tid; e < TT; e += CTH) A.Lg[(size_t)t * TT + e] = T[e];
        }
        int any_bad = 0;
        cl.sync();
        for (int rk = 0; rk < CL; rk++) any_bad |= *cl.map_shared_rank(&bad, rk);
        cl.sync();  // nobody leaves while another CTA may still read its flag
        if (any_bad) {
            if (rank == 0 && tid == 0) {
                A.flags[0] = 0;
                A.flags[2] = (int)SFFT_ERR_NOT_SPD;
            }
            return;
        }
    }

    // ---------------------------------------------------------------- preconditioner apply
    // v <- (L L^T)^{-1} v on every CTA's copy of v (the vector is broadcast block by block)
    auto precond = [&]() {
        // forward: L y = v
        for (int kb = 0; kb < nblk; kb++) {
            const int td = tile_id(kb, kb);
            if (owner(td) == rank) {
                const float *a = local(td);
                if (tid < 32) {
                    float yr = v[kb * TB + tid];
                    for (int c = 0; c < TB; c++) {
                        float yc = __shfl_sync(0xffffffffu, yr, c) * a[c * TS + TB];
                        if (tid == c) yr = yc;
                        if (tid > c) yr -= a[tid * TS + c] * yc;
                    }
                    for (int rk = 0; rk < CL; rk++) cl.map_shared_rank(v, rk)[kb * TB + tid] = yr;
                }
            }
            cl.sync();
            for (int ib = kb + 1; ib < nblk; ib++) {
                const int t = tile_id(ib, kb);
                if (owner(t) != rank || tid >= 32) continue;
                const float *a = local(t);
                float s = 0.0f;
                for (int c = 0; c < TB; c++) s += a[tid * TS + c] * v[kb * TB + c];
                float *dst = cl.map_shared_rank(v, owner(tile_id(ib, ib)));
                dst[ib * TB + tid] -= s;
            }
            cl.sync();
        }
        // backward: L^T x = y
        for (int kb = nblk - 1; kb >= 0; kb--) {
            const int td = tile_id(kb, kb);
            if (owner(td) == rank) {
                const float *a = local(td);
                if (tid < 32) {
                    float xr = v[kb * TB + tid];
                    for (int c = TB - 1; c >= 0; c--) {
                        float xc = __shfl_sync(0xffffffffu, xr, c) * a[c * TS + TB];
                        if (tid == c) xr = xc;
                        if (tid < c) xr -= a[c * TS + tid] * xc;
                    }
                    for (int rk = 0; rk < CL; rk++) cl.map_shared_rank(v, rk)[kb * TB + tid] = xr;
                }
            }
            cl.sync();
            for (int jb = 0; jb < kb; jb++) {
                const int t = tile_id(kb, jb);
                if (owner(t) != rank || tid >= 32) continue;
                const float *a = local(t);
                float s = 0.0f;
                for (int rr = 0; rr < TB; rr++) s += a[rr * TS + tid] * v[kb * TB + rr];
                float *dst = cl.map_shared_rank(v, owner(tile_id(jb, jb)));
                dst[jb * TB + tid] -= s;
            }
            cl.sync();
        }
    };
    const int gw = rank * (CTH / 32) + (tid >> 5), nw = CL * (CTH / 32), lane = tid & 31;
    // z = D (L L^T)^{-1} D r, using v as the FP32 work vector
    auto apply_M = [&](const double *rvec, double *zvec) {
        for (int i = tid; i < npad; i += CTH) v[i] = i < n ? (float)(__ldcg(A.d + i) * __ldcg(rvec + i)) : 0.0f;
        cl.sync();
        precond();
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) zvec[i] = __ldcg(A.d + i) * (double)v[i];
        cl.sync();
    };

    if (A.mode == 1) {
        // one correction with the stored factor: x += M^{-1} c
        apply_M(A.b, A.z);
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) A.x[i] += A.z[i];
        return;
    }

    // ---------------------------------------------------------------- PCG in FP64
    // rows of N are distributed one warp per row over the cluster
    auto matvec = [&](const double *xin, double *yout) {
        for (int i = gw; i < n; i += nw) {
            const double *row = A.N + (size_t)i * n;
            double s = 0.0;
            for (int j = lane; j < n; j += 32) s = fma(row[j], __ldcg(xin + j), s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) yout[i] = s;
        }
    };
    auto dot = [&](const double *u, const double *w) {
        double s = 0.0;
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) s += __ldcg(u + i) * __ldcg(w + i);
        return cluster_sum(cl, &slot, s);
    };
    // x0: Galerkin projection onto span{x0, background unit vectors}, or zero
    __shared__ double gal[kGalMax * (kGalMax + 1)], gco[kGalMax];
    if (A.x0) {
        matvec(A.x0, A.q);
        cl.sync();
        const double xq = dot(A.x0, A.q), xb = dot(A.x0, A.b);
        const int m = A.nb + 1 <= kGalMax ? A.nb + 1 : 1;
        if (threadIdx.x == 0) {
            // order (x0, e_0, e_1, ...): G_00 = x0.N x0, G_0r = (N x0)_r, G_rs = N_rs
            for (int i = 0; i < m; i++) {
                for (int j = 0; j < m; j++) {
                    double v;
                    if (i == 0 && j == 0)
                        v = xq;
                    else if (i == 0)
                        v = __ldcg(A.q + A.nker + j - 1);
                    else if (j == 0)
                        v = __ldcg(A.q + A.nker + i - 1);
                    else
                        v = A.N[(size_t)(A.nker + i - 1) * n + A.nker + j - 1];
                    gal[i * (m + 1) + j] = v;
                }
                gal[i * (m + 1) + m] = i == 0 ? xb : A.b[A.nker + i - 1];
            }
            solve_small(gal, m, gco);
        }
        __syncthreads();
        // x = alpha x0 + sum_r beta_r e_r; its residual r = b - N x from the products already
        // at hand (N x = alpha N x0 + sum_r beta_r N e_r, the background columns of N), so
        // the warm start costs one matrix-vector product, not two
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) {
            const int rr = i - A.nker;
            A.x[i] = gco[0] * A.x0[i] + (rr >= 0 && rr < m - 1 ? gco[1 + rr] : 0.0);
            double nxi = gco[0] * __ldcg(A.q + i);
            for (int k = 1; k < m; k++) nxi = fma(gco[k], A.N[(size_t)i * n + A.nker + k - 1], nxi);
            A.r[i] = A.b[i] - nxi;
        }
    } else {
        // cold start: x = 0 and r = b, no product needed
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) {
            A.x[i] = 0.0;
            A.r[i] = A.b[i];
        }
    }
    cl.sync();
    const double bb = dot(A.b, A.b);
    apply_M(A.r, A.z);
    for (int i = rank * CTH + tid; i < n; i += CL * CTH) A.p[i] = __ldcg(A.z + i);
    cl.sync();
    double rz = dot(A.r, A.z), rr = dot(A.r, A.r);
    const double rr0 = rr;
    int it = 0;
    bool conv = rr <= A.tol * A.tol * bb;
    while (!conv && it < A.max_iter && isfinite(rz)) {
        matvec(A.p, A.q);
        cl.sync();
        const double pq = dot(A.p, A.q);
        if (!(pq > 0.0)) break;
        const double alpha = rz / pq;
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) {
            A.x[i] = __ldcg(A.x + i) + alpha * __ldcg(A.p + i);
            A.r[i] = __ldcg(A.r + i) - alpha * __ldcg(A.q + i);
        }
        cl.sync();
        it++;
        rr = dot(A.r, A.r);
        if (rr <= A.tol * A.tol * bb) {
            conv = true;
            break;
        }
        apply_M(A.r, A.z);
        const double rz_new = dot(A.r, A.z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int i = rank * CTH + tid; i < n; i += CL * CTH) A.p[i] = __ldcg(A.z + i) + beta * __ldcg(A.p + i);
        cl.sync();
    }
    if (rank == 0 && tid == 0) {
        A.flags[0] = conv ? 1 : 0;
        A.flags[1] = it;
        // why PCG stopped short: the iteration cap, or a breakdown (p^T N p <= 0, NaN)
        A.flags[2] = conv ? 0 : (it >= A.max_iter ? (int)SFFT_ERR_NO_CONVERGENCE : (int)SFFT_ERR_NOT_SPD);
        A.scal[0] = rr;
        A.scal[1] = bb;
        A.scal[2] = rr0;
    }
}

int g_cluster = -1;  // chosen cluster size (0: unavailable)

size_t pcg_smem(int ntiles, int nblk, int CL) {
    const int ntl = (ntiles + CL - 1) / CL;
    return sizeof(float) * ((size_t)ntl * TT + 3 * TT + (size_t)nblk * TB);
}

}  // namespace

int pcg_cluster_size(const Geometry &g) {
    const int nblk = (g.n + TB - 1) / TB, ntiles = nblk * (nblk + 1) / 2;
    if (g_cluster < 0) {
        g_cluster = 0;
        for (int CL : {16, 8}) {
            cudaError_t e = cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            size_t sm = 200 * 1024;
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CL);
            cfg.blockDim = dim3(CTH);
            cfg.dynamicSmemBytes = sm;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = CL;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            e = cudaOccupancyMaxActiveClusters(&nclusters, k_pcg_cluster, &cfg);
            if (e == cudaSuccess && nclusters > 0) {
                g_cluster = CL;
                break;
            }
            cudaGetLastError();
        }
    }
    if (g_cluster == 0) return 0;
    const int CL = g.pcg_cluster > 0 && g.pcg_cluster < g_cluster ? g.pcg_cluster : g_cluster;
    if (pcg_smem(ntiles, nblk, CL) > 200 * 1024) return 0;  // factor does not fit: no fast path
    return CL;
}

size_t pcg_factor_floats(const Geometry &g) {
    const int nblk = (g.n + TB - 1) / TB;
    return (size_t)nblk * (nblk + 1) / 2 * TT;
}

cudaError_t launch_pcg_cluster(const Geometry &g, const double *N, const double *b, const double *x0, double *x,
                               double *r, double *p, double *q, double *z, double *d, float *Lg, double *scal,
                               int *flags, int max_iter, double tol, bool correction, cudaStream_t st) {
    const int CL = pcg_cluster_size(g);
    if (CL == 0) return cudaErrorNotSupported;
    FastArgs A;
    A.N = N;
    A.b = b;
    A.x0 = x0;
    A.nker = g.nker;
    A.nb = g.nb;
    A.x = x;
    A.r = r;
    A.p = p;
    A.q = q;
    A.z = z;
    A.d = d;
    A.Lg = Lg;
    A.scal = scal;
    A.flags = flags;
    A.n = g.n;
    A.nblk = (g.n + TB - 1) / TB;
    A.ntiles = A.nblk * (A.nblk + 1) / 2;
    A.max_iter = max_iter;
    A.tol = tol;
    A.mode = correction ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(CTH);
    cfg.dynamicSmemBytes = pcg_smem(A.ntiles, A.nblk, CL);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k_pcg_cluster, A);
}

}  // namespace sfft
