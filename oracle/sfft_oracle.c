/*
 * FP64 CPU oracle for the SFFT fit and subtraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code with the CUDA library.
 *
 * What it computes (the SFFT subtraction step of the pipeline, Sec. "Pipeline steps",
 * step 6; a delta-basis matching kernel that can follow a spatially varying PSF,
 * Sec. "Statement of need"; "the large linear system it solves", Sec. "Future
 * development").  The paper prints no equations for the method, so the statement
 * below is the least-squares problem written out from first principles:
 *
 *   frame Ny x Nx, pixel u = (y, x), row-major; normalised coordinates
 *     xh = 2x/(Nx-1) - 1, yh = 2y/(Ny-1) - 1   (0 when the axis has one pixel);
 *   monomials w_pq = xh^p yh^q, p+q <= D, ordered by total degree, then q ascending;
 *   mask m(u) = 1 for good pixels, 0 where the mask byte is non-zero;
 *   X_m = m * X;  cyclic shift (X(. - d))(u) = X((u - d) mod N);
 *   kernel basis  Phi_{pq,d}(u) = W_pq((u - d) mod N),  W_pq = w_pq * T_m,
 *                 p+q <= DK, lag d = (dx, dy) in [-h, h]^2, h = (L-1)/2,
 *                 d ordered row-major (dy outer);
 *   background    Psi_rs = m * w_rs, r+s <= DB;
 *   unknowns      theta = [a_{pq,d} (pq-major blocks of L^2 lags); b_rs];
 *   normal eqs    N = [Phi Psi]^T [Phi Psi],  b = [Phi Psi]^T S_m;  N theta = b;
 *   difference    D(u) = S(u) - sum a_{pq,d} (w_pq T)((u - d) mod N) - sum b_rs w_rs(u).
 *
 * Steps, in order:
 *   1. cast to FP64, form W_pq, S_m, Psi_rs (and w_pq T for the difference image);
 *   2. lag tables by direct spatial sums with Neumaier-compensated accumulation,
 *        C_AB(D) = sum_u A(u) B((u + D) mod N),
 *      using  <Phi_{pq,d}, Phi_{p'q',d'}> = C_{W_pq,W_p'q'}(d - d'),
 *             <Phi_{pq,d}, Psi_rs>       = C_{W_pq,Psi_rs}(d),
 *             <Phi_{pq,d}, S_m>          = C_{W_pq,S_m}(d);
 *   3. assemble N and b from the tables (symmetric by construction);
 *   4. plain right-looking FP64 Cholesky, no pivoting, then two triangular solves;
 *   5. D by direct spatial sums.
 * A second, independent route (oracle_brute_normal) materialises every basis image
 * and forms each entry of N and b as a dot product; oracle_normal_entries evaluates
 * single entries the same way at any frame size.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 3
#define OR_ERR_NOT_SPD 4

/* ------------------------------------------------------------------ helpers */

typedef struct {
    double s, c;
} nsum_t; /* Neumaier running sum: value = s + c */

static inline void nsum_add(nsum_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nsum_val(const nsum_t *a) { return a->s + a->c; }

int oracle_npoly(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

/* exponents (p, q) of monomial number idx: total degree first, then q ascending */
void oracle_mono_pq(int idx, int *p, int *q) {
    int d = 0;
    while (idx > d) {
        idx -= d + 1;
        d++;
    }
    *q = idx;
    *p = d - idx;
}

static double coord(int i, int n) { return n > 1 ? 2.0 * (double)i / (double)(n - 1) - 1.0 : 0.0; }

static double ipow(double v, int e) {
    double r = 1.0;
    for (int k = 0; k < e; k++) r *= v;
    return r;
}

static double mono_at(int idx, int y, int x, int ny, int nx) {
    int p, q;
    oracle_mono_pq(idx, &p, &q);
    return ipow(coord(x, nx), p) * ipow(coord(y, ny), q);
}

static inline int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static int check_args(int ny, int nx, int L, int dk, int db) {
    if (ny < 1 || nx < 1 || L < 1 || (L % 2) == 0 || dk < 0 || db < 0) return OR_ERR_ARG;
    if (ny < L || nx < L) return OR_ERR_ARG;
    return OR_OK;
}

int oracle_n_unknowns(int L, int dk, int db) { return L * L * oracle_npoly(dk) + oracle_npoly(db); }

/* Step 1: FP64 basis images.  img layout: [W_0..W_{nk-1}, G_0..G_{nb-1}, S_m] each ny*nx. */
static double *make_basis(int ny, int nx, const double *S, const double *T, const uint8_t *mask,
                          int dk, int db) {
    int nk = oracle_npoly(dk), nb = oracle_npoly(db);
    size_t np = (size_t)ny * nx;
    double *img = (double *)malloc(sizeof(double) * np * (size_t)(nk + nb + 1));
    if (!img) return NULL;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++) {
        for (int x = 0; x < nx; x++) {
            size_t u = (size_t)y * nx + x;
            double m = (mask && mask[u]) ? 0.0 : 1.0;
            /* a masked pixel is zero in the fit whatever it holds (NaN included) */
            double tm = m != 0.0 ? T[u] : 0.0, sm = m != 0.0 ? S[u] : 0.0;
            for (int i = 0; i < nk; i++) img[(size_t)i * np + u] = mono_at(i, y, x, ny, nx) * tm;
            for (int r = 0; r < nb; r++) img[(size_t)(nk + r) * np + u] = mono_at(r, y, x, ny, nx) * m;
            img[(size_t)(nk + nb) * np + u] = sm;
        }
    }
    return img;
}

/* C_AB(dx, dy) = sum_u A(u) B((u + d) mod N), Neumaier-compensated. */
static double corr(const double *A, const double *B, int ny, int nx, int dx, int dy) {
    nsum_t acc = {0.0, 0.0};
    for (int y = 0; y < ny; y++) {
        const double *a = A + (size_t)y * nx;
        const double *b = B + (size_t)wrap(y + dy, ny) * nx;
        for (int x = 0; x < nx; x++) {
            int xb = x + dx; /* |dx| < nx, so one correction wraps it */
            if (xb >= nx) xb -= nx;
            else if (xb < 0) xb += nx;
            nsum_add(&acc, a[x] * b[xb]);
        }
    }
    return nsum_val(&acc);
}

static int pair_index(int i, int j, int nk) { /* i <= j, row-major upper triangle */
    return i * nk - i * (i - 1) / 2 + (j - i);
}

/* ------------------------------------------------------------ step 2: lag tables */

/*
 * Lag tables.
 *   Cww[pair(i,j)][dy + L-1][dx + L-1] = C_{W_i,W_j}(dx,dy), i <= j, |dx|,|dy| <= L-1
 *   Cwg[i][r][dy + h][dx + h]          = C_{W_i,Psi_r}(dx,dy),   |dx|,|dy| <= h
 *   Cws[i][dy + h][dx + h]             = C_{W_i,S_m}(dx,dy),     |dx|,|dy| <= h
 *   Ggg[r][r'] = sum_u Psi_r Psi_r',   Ggs[r] = sum_u Psi_r S_m
 */
int oracle_lag_tables(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L,
                      int dk, int db, double *Cww, double *Cwg, double *Cws, double *Ggg,
                      double *Ggs) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    int nk = oracle_npoly(dk), nb = oracle_npoly(db), h = (L - 1) / 2;
    int Lw = 2 * L - 1, nww = Lw * Lw, ns = L * L;
    int npair = nk * (nk + 1) / 2;
    size_t np = (size_t)ny * nx;
    double *img = make_basis(ny, nx, S, T, mask, dk, db);
    if (!img) return OR_ERR_OOM;
    const double *W = img, *G = img + (size_t)nk * np, *Sm = img + (size_t)(nk + nb) * np;

    long n_ww = (long)npair * nww, n_wg = (long)nk * nb * ns, n_ws = (long)nk * ns;
    long total = n_ww + n_wg + n_ws;
#pragma omp parallel for schedule(dynamic, 1)
    for (long e = 0; e < total; e++) {
        if (e < n_ww) {
            int pr = (int)(e / nww), l = (int)(e % nww);
            int i = 0, j = 0;
            for (int a = 0, c = 0; a < nk; a++)
                for (int b2 = a; b2 < nk; b2++, c++)
                    if (c == pr) { i = a; j = b2; }
            int dy = l / Lw - (L - 1), dx = l % Lw - (L - 1);
            Cww[e] = corr(W + (size_t)i * np, W + (size_t)j * np, ny, nx, dx, dy);
        } else if (e < n_ww + n_wg) {
            long f = e - n_ww;
            int i = (int)(f / ((long)nb * ns)), r = (int)((f / ns) % nb), l = (int)(f % ns);
            int dy = l / L - h, dx = l % L - h;
            Cwg[f] = corr(W + (size_t)i * np, G + (size_t)r * np, ny, nx, dx, dy);
        } else {
            long f = e - n_ww - n_wg;
            int i = (int)(f / ns), l = (int)(f % ns);
            int dy = l / L - h, dx = l % L - h;
            Cws[f] = corr(W + (size_t)i * np, Sm, ny, nx, dx, dy);
        }
    }
    for (int r = 0; r < nb; r++) {
        for (int r2 = 0; r2 < nb; r2++) Ggg[r * nb + r2] = corr(G + (size_t)r * np, G + (size_t)r2 * np, ny, nx, 0, 0);
        Ggs[r] = corr(G + (size_t)r * np, Sm, ny, nx, 0, 0);
    }
    free(img);
    return OR_OK;
}

/*
 * The same lag tables restricted to the rows y0 <= y < y1 of the first factor:
 *   C^band_AB(D) = sum_{y0 <= y < y1} sum_x A(y, x) B((y + dy) mod ny, (x + dx) mod nx).
 * The tables of bands that cover [0, ny) add up to the full tables (the sums of step 2,
 * split by rows).  Only the rows a band reads are formed: y0 - (L-1) .. y1 + (L-1) - 1,
 * taken modulo ny.  Used to time the oracle on one full frame in slices.
 */
int oracle_lag_tables_band(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L,
                           int dk, int db, int y0, int y1, double *Cww, double *Cwg, double *Cws,
                           double *Ggg, double *Ggs) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    if (y0 < 0 || y1 > ny || y0 >= y1) return OR_ERR_ARG;
    int nk = oracle_npoly(dk), nb = oracle_npoly(db), h = (L - 1) / 2;
    int Lw = 2 * L - 1, nww = Lw * Lw, ns = L * L, G = L - 1;
    int npair = nk * (nk + 1) / 2;
    int nrow = (y1 - y0) + 2 * G; /* local row r is frame row (y0 - G + r) mod ny */
    size_t np = (size_t)nrow * nx;
    int nimg = nk + nb + 1;
    double *img = (double *)malloc(sizeof(double) * np * (size_t)nimg);
    if (!img) return OR_ERR_OOM;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nrow; r++) {
        int y = wrap(y0 - G + r, ny);
        for (int x = 0; x < nx; x++) {
            size_t u = (size_t)y * nx + x, v = (size_t)r * nx + x;
            double m = (mask && mask[u]) ? 0.0 : 1.0;
            double tm = m != 0.0 ? T[u] : 0.0, sm = m != 0.0 ? S[u] : 0.0;
            for (int i = 0; i < nk; i++) img[(size_t)i * np + v] = mono_at(i, y, x, ny, nx) * tm;
            for (int q = 0; q < nb; q++) img[(size_t)(nk + q) * np + v] = mono_at(q, y, x, ny, nx) * m;
            img[(size_t)(nk + nb) * np + v] = sm;
        }
    }
    const double *W = img, *Gb = img + (size_t)nk * np, *Sm = img + (size_t)(nk + nb) * np;
    const int nband = y1 - y0;
    long n_ww = (long)npair * nww, n_wg = (long)nk * nb * ns, n_ws = (long)nk * ns;
    long n_gg = (long)nb * nb, n_gs = nb;
    long total = n_ww + n_wg + n_ws + n_gg + n_gs;
#pragma omp parallel for schedule(dynamic, 1)
    for (long e = 0; e < total; e++) {
        const double *A, *B;
        int dx = 0, dy = 0;
        double *out;
        if (e < n_ww) {
            int pr = (int)(e / nww), l = (int)(e % nww), i = 0, j = 0;
            for (int a = 0, c = 0; a < nk; a++)
                for (int b2 = a; b2 < nk; b2++, c++)
                    if (c == pr) { i = a; j = b2; }
            dy = l / Lw - (L - 1);
            dx = l % Lw - (L - 1);
            A = W + (size_t)i * np;
            B = W + (size_t)j * np;
            out = Cww + e;
        } else if (e < n_ww + n_wg) {
            long f = e - n_ww;
            int i = (int)(f / ((long)nb * ns)), q = (int)((f / ns) % nb), l = (int)(f % ns);
            dy = l / L - h;
            dx = l % L - h;
            A = W + (size_t)i * np;
            B = Gb + (size_t)q * np;
            out = Cwg + f;
        } else if (e < n_ww + n_wg + n_ws) {
            long f = e - n_ww - n_wg;
            int i = (int)(f / ns), l = (int)(f % ns);
            dy = l / L - h;
            dx = l % L - h;
            A = W + (size_t)i * np;
            B = Sm;
            out = Cws + f;
        } else if (e < n_ww + n_wg + n_ws + n_gg) {
            long f = e - n_ww - n_wg - n_ws;
            A = Gb + (size_t)(f / nb) * np;
            B = Gb + (size_t)(f % nb) * np;
            out = Ggg + f;
        } else {
            long f = e - n_ww - n_wg - n_ws - n_gg;
            A = Gb + (size_t)f * np;
            B = Sm;
            out = Ggs + f;
        }
        nsum_t acc = {0.0, 0.0};
        for (int yy = 0; yy < nband; yy++) {
            const double *a = A + (size_t)(G + yy) * nx;
            const double *b = B + (size_t)(G + yy + dy) * nx;
            for (int x = 0; x < nx; x++) {
                int xb = x + dx;
                if (xb >= nx) xb -= nx;
                else if (xb < 0) xb += nx;
                nsum_add(&acc, a[x] * b[xb]);
            }
        }
        *out = nsum_val(&acc);
    }
    free(img);
    return OR_OK;
}

/* ---------------------------------------------------------- step 3: assembly */

int oracle_assemble(int L, int dk, int db, const double *Cww, const double *Cwg, const double *Cws,
                    const double *Ggg, const double *Ggs, double *N, double *b) {
    if (L < 1 || (L % 2) == 0 || dk < 0 || db < 0) return OR_ERR_ARG;
    int nk = oracle_npoly(dk), nb = oracle_npoly(db), h = (L - 1) / 2;
    int Lw = 2 * L - 1, ns = L * L, nker = nk * ns, n = nker + nb;
    for (int i = 0; i < nk; i++)
        for (int l = 0; l < ns; l++) {
            int row = i * ns + l, dy = l / L - h, dx = l % L - h;
            for (int j = 0; j < nk; j++)
                for (int l2 = 0; l2 < ns; l2++) {
                    int col = j * ns + l2, dy2 = l2 / L - h, dx2 = l2 % L - h;
                    /* <Phi_{i,d}, Phi_{j,d'}> = C_{W_i,W_j}(d - d') = C_{W_j,W_i}(d' - d) */
                    double v;
                    if (i <= j)
                        v = Cww[(size_t)pair_index(i, j, nk) * Lw * Lw + (size_t)(dy - dy2 + L - 1) * Lw + (dx - dx2 + L - 1)];
                    else
                        v = Cww[(size_t)pair_index(j, i, nk) * Lw * Lw + (size_t)(dy2 - dy + L - 1) * Lw + (dx2 - dx + L - 1)];
                    N[(size_t)row * n + col] = v;
                }
            for (int r = 0; r < nb; r++) {
                double v = Cwg[((size_t)i * nb + r) * ns + l];
                N[(size_t)row * n + nker + r] = v;
                N[(size_t)(nker + r) * n + row] = v;
            }
            b[row] = Cws[(size_t)i * ns + l];
        }
    for (int r = 0; r < nb; r++) {
        for (int r2 = 0; r2 < nb; r2++) N[(size_t)(nker + r) * n + nker + r2] = Ggg[r * nb + r2];
        b[nker + r] = Ggs[r];
    }
    return OR_OK;
}

int oracle_normal(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L,
                  int dk, int db, double *N, double *b) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    int nk = oracle_npoly(dk), nb = oracle_npoly(db), Lw = 2 * L - 1;
    int npair = nk * (nk + 1) / 2;
    double *Cww = (double *)malloc(sizeof(double) * (size_t)npair * Lw * Lw);
    double *Cwg = (double *)malloc(sizeof(double) * (size_t)nk * nb * L * L + 1);
    double *Cws = (double *)malloc(sizeof(double) * (size_t)nk * L * L);
    double *Ggg = (double *)malloc(sizeof(double) * (size_t)nb * nb + 1);
    double *Ggs = (double *)malloc(sizeof(double) * (size_t)nb + 1);
    if (!Cww || !Cwg || !Cws || !Ggg || !Ggs) rc = OR_ERR_OOM;
    if (!rc) rc = oracle_lag_tables(ny, nx, S, T, mask, L, dk, db, Cww, Cwg, Cws, Ggg, Ggs);
    if (!rc) rc = oracle_assemble(L, dk, db, Cww, Cwg, Cws, Ggg, Ggs, N, b);
    free(Cww); free(Cwg); free(Cws); free(Ggg); free(Ggs);
    return rc;
}

/* ------------------------------------------- independent route: brute force */

/* value of basis function k (0..n-1) at pixel (y, x); k == n means S_m */
static double basis_value(int k, int y, int x, int ny, int nx, const double *S, const double *T,
                          const uint8_t *mask, int L, int dk, int db) {
    int nk = oracle_npoly(dk), ns = L * L, h = (L - 1) / 2, nker = nk * ns;
    (void)db;
    if (k < nker) {
        int i = k / ns, l = k % ns, dy = l / L - h, dx = l % L - h;
        int ys = wrap(y - dy, ny), xs = wrap(x - dx, nx);
        size_t u = (size_t)ys * nx + xs;
        if (mask && mask[u]) return 0.0;
        return mono_at(i, ys, xs, ny, nx) * T[u];
    }
    size_t u = (size_t)y * nx + x;
    if (mask && mask[u]) return 0.0;
    if (k < nker + oracle_npoly(db)) return mono_at(k - nker, y, x, ny, nx);
    return S[u];
}

/* N and b as explicit dot products of materialised basis images (tiny frames only). */
int oracle_brute_normal(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L,
                        int dk, int db, double *N, double *b) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    int n = oracle_n_unknowns(L, dk, db);
    size_t np = (size_t)ny * nx;
    double *B = (double *)malloc(sizeof(double) * np * (size_t)(n + 1));
    if (!B) return OR_ERR_OOM;
    for (int k = 0; k <= n; k++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                B[(size_t)k * np + (size_t)y * nx + x] = basis_value(k, y, x, ny, nx, S, T, mask, L, dk, db);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n; r++) {
        for (int c = 0; c <= n; c++) {
            nsum_t acc = {0.0, 0.0};
            for (size_t u = 0; u < np; u++) nsum_add(&acc, B[(size_t)r * np + u] * B[(size_t)c * np + u]);
            if (c < n)
                N[(size_t)r * n + c] = nsum_val(&acc);
            else
                b[r] = nsum_val(&acc);
        }
    }
    free(B);
    return OR_OK;
}

/* Single entries by definition, at any frame size: out[e] = <basis_rows[e], basis_cols[e]>,
 * where column index n selects S_m (so the entry is b[row]). */
int oracle_normal_entries(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L,
                          int dk, int db, int n_entries, const int64_t *rows, const int64_t *cols,
                          double *out) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    int n = oracle_n_unknowns(L, dk, db);
    for (int e = 0; e < n_entries; e++)
        if (rows[e] < 0 || rows[e] >= n || cols[e] < 0 || cols[e] > n) return OR_ERR_ARG;
    for (int e = 0; e < n_entries; e++) {
        double s = 0.0, c = 0.0;
#pragma omp parallel
        {
            nsum_t acc = {0.0, 0.0};
#pragma omp for schedule(static)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++)
                    nsum_add(&acc, basis_value((int)rows[e], y, x, ny, nx, S, T, mask, L, dk, db) *
                                       basis_value((int)cols[e], y, x, ny, nx, S, T, mask, L, dk, db));
#pragma omp critical
            {
                nsum_t tot = {s, c};
                nsum_add(&tot, acc.s);
                nsum_add(&tot, acc.c);
                s = tot.s;
                c = tot.c;
            }
        }
        out[e] = s + c;
    }
    return OR_OK;
}

/* ------------------------------------------------------------- step 4: solve */

/* N = R^T R with R upper triangular (plain right-looking FP64 Cholesky, no pivoting),
 * then R^T z = b, R x = z.  Returns OR_ERR_NOT_SPD on a non-positive pivot. */
int oracle_cholesky_solve(int n, const double *N, const double *b, double *x) {
    if (n < 1) return OR_ERR_ARG;
    double *R = (double *)malloc(sizeof(double) * (size_t)n * n);
    if (!R) return OR_ERR_OOM;
    memcpy(R, N, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < n; k++) {
        double d = R[(size_t)k * n + k];
        if (!(d > 0.0) || !isfinite(d)) {
            free(R);
            return OR_ERR_NOT_SPD;
        }
        d = sqrt(d);
        R[(size_t)k * n + k] = d;
        for (int j = k + 1; j < n; j++) R[(size_t)k * n + j] /= d;
        /* trailing update of the upper triangle: A[i][j] -= R[k][i] R[k][j] */
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int i = k + 1; i < n; i++) {
            double rki = R[(size_t)k * n + i];
            for (int j = i; j < n; j++) R[(size_t)i * n + j] -= rki * R[(size_t)k * n + j];
        }
    }
    for (int i = 0; i < n; i++) { /* R^T z = b */
        double s = b[i];
        for (int k = 0; k < i; k++) s -= R[(size_t)k * n + i] * x[k];
        x[i] = s / R[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) { /* R x = z */
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= R[(size_t)i * n + k] * x[k];
        x[i] = s / R[(size_t)i * n + i];
    }
    free(R);
    return OR_OK;
}

int oracle_fit(int ny, int nx, const double *S, const double *T, const uint8_t *mask, int L, int dk,
               int db, double *theta) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    int n = oracle_n_unknowns(L, dk, db);
    double *N = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    if (!N || !b) rc = OR_ERR_OOM;
    if (!rc) rc = oracle_normal(ny, nx, S, T, mask, L, dk, db, N, b);
    if (!rc) rc = oracle_cholesky_solve(n, N, b, theta);
    free(N);
    free(b);
    return rc;
}

/* ------------------------------------------------- step 5: difference image */

static double diff_pixel(int y, int x, int ny, int nx, const double *S, const double *T, int L,
                         int dk, int db, const double *theta) {
    int nk = oracle_npoly(dk), nb = oracle_npoly(db), ns = L * L, h = (L - 1) / 2;
    nsum_t acc = {0.0, 0.0};
    nsum_add(&acc, S[(size_t)y * nx + x]);
    for (int i = 0; i < nk; i++)
        for (int l = 0; l < ns; l++) {
            int dy = l / L - h, dx = l % L - h;
            int ys = wrap(y - dy, ny), xs = wrap(x - dx, nx);
            nsum_add(&acc, -theta[i * ns + l] * mono_at(i, ys, xs, ny, nx) * T[(size_t)ys * nx + xs]);
        }
    for (int r = 0; r < nb; r++) nsum_add(&acc, -theta[nk * ns + r] * mono_at(r, y, x, ny, nx));
    return nsum_val(&acc);
}

int oracle_subtract(int ny, int nx, const double *S, const double *T, int L, int dk, int db,
                    const double *theta, double *D) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) D[(size_t)y * nx + x] = diff_pixel(y, x, ny, nx, S, T, L, dk, db, theta);
    return OR_OK;
}

/* D at selected pixels (flat row-major indices), for sampled checks on large frames. */
int oracle_subtract_pixels(int ny, int nx, const double *S, const double *T, int L, int dk, int db,
                           const double *theta, int n_pix, const int64_t *idx, double *out) {
    int rc = check_args(ny, nx, L, dk, db);
    if (rc) return rc;
    for (int e = 0; e < n_pix; e++)
        if (idx[e] < 0 || idx[e] >= (int64_t)ny * nx) return OR_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < n_pix; e++)
        out[e] = diff_pixel((int)(idx[e] / nx), (int)(idx[e] % nx), ny, nx, S, T, L, dk, db, theta);
    return OR_OK;
}

/* ------------------------------------------ cross-convolution (pipeline step 5) */

/* out(u) = sum_d P(d) X((u - d) mod N), d = (a - r, b - r) for the K x K stamp P[a][b]
 * (K = 2r + 1, row-major): the cyclic convolution of the image with the stamp, centred on
 * the stamp's middle element, by direct FP64 sums. */
int oracle_convolve(int ny, int nx, const double *X, int K, const double *P, double *out) {
    if (ny < 1 || nx < 1 || K < 1 || (K % 2) == 0) return OR_ERR_ARG;
    int r = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            nsum_t acc = {0.0, 0.0};
            for (int a = 0; a < K; a++)
                for (int b = 0; b < K; b++)
                    nsum_add(&acc, P[a * K + b] * X[(size_t)wrap(y - (a - r), ny) * nx + wrap(x - (b - r), nx)]);
            out[(size_t)y * nx + x] = nsum_val(&acc);
        }
    return OR_OK;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
