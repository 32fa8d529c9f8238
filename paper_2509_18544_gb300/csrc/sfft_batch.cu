// Batches of science/template pairs (the S x T pairing of Sec. "Pipeline steps", step 1)
// and the launch-shape tuning cache.
//
// Batch executor.  Pairs are spread over `lanes` CUDA streams by longest-processing-time
// first (cost ~ pixels plus a constant for the solve), each lane owning one plan per
// distinct geometry it meets, so one pair's latency-bound solve overlaps other pairs'
// FFT and correlation stages.  After each fit the plan's device status, solver flags and
// residual norms are copied into a per-pair record and the status word is cleared, so
// every pair reports its own outcome.  With SFFT_BATCH_GRAPH the whole batch -- fork into
// the lanes, every fit and subtraction, the records, the join -- is captured once into a
// CUDA graph and each run is a single graph launch on the caller's stream.
//
// Tuning cache.  A plan's y-correlation shape (frequencies per CTA, row chunks, packed or
// scalar FP32 kernel) and the subtract grid density come from a process-wide table keyed by
// the descriptor; sfft_autotune fills an entry by timing candidate shapes on real data
// (coordinate descent, CUDA events on the plan's stream).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "sfft_internal.cuh"

namespace sfft {
void set_global_error(const char *msg);
void finish_geometry(Geometry &g);
}

using namespace sfft;

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int, int, int>;

Key key_of(const sfft_desc &d) {
    return Key(d.ny, d.nx, d.pitch ? d.pitch : d.nx, d.L, d.dk, d.db, d.dtype, d.precision, d.solver, d.refine);
}

std::mutex g_tune_mu;
std::map<Key, sfft_tuning> g_tune;

void errf(const char *fmt, ...) __attribute__((format(printf, 1, 2)));
void errf(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
}

// checks a tuning against the geometry's limits and applies it
bool apply_tuning(const sfft_tuning &t, Geometry &g, char *err, size_t errlen) {
    if (t.ycorr_bins < 0 || t.ycorr_bins > g.kg_max)
        return snprintf(err, errlen, "ycorr_bins %d outside [0, %d]", t.ycorr_bins, g.kg_max), false;
    if (t.ycorr_bins > 0) g.kg = t.ycorr_bins;
    if (t.ycorr_direct != 0 && t.ycorr_direct != 1) return snprintf(err, errlen, "ycorr_direct must be 0 or 1"), false;
    if (t.ycorr_direct) g.yfft = 0;
    const int max_ys = g.yfft ? 64 : std::max(1, g.ny / (2 * g.ytile));
    if (t.ycorr_split < 0 || t.ycorr_split > max_ys)
        return snprintf(err, errlen, "ycorr_split %d outside [0, %d]", t.ycorr_split, max_ys), false;
    if (g.yfft) {
        if (t.ycorr_split > 0) g.y2split = t.ycorr_split;
    } else {
        g.ysplit = t.ycorr_split > 0 ? t.ycorr_split : default_ysplit(g);
    }
    finish_geometry(g);
    if (t.ycorr_sets < 0 || t.ycorr_sets > 2) return snprintf(err, errlen, "ycorr_sets must be 0, 1 or 2"), false;
    if (t.ycorr_sets > 0) g.ysets = t.ycorr_sets;
    if (t.ycorr_scalar != 0 && t.ycorr_scalar != 1) return snprintf(err, errlen, "ycorr_scalar must be 0 or 1"), false;
    g.ycorr_scalar = t.ycorr_scalar;
    if (t.subtract_ctas < 0 || t.subtract_ctas > 4)
        return snprintf(err, errlen, "subtract_ctas %d outside [0, 4]", t.subtract_ctas), false;
    g.sub_per_sm = t.subtract_ctas > 0 ? t.subtract_ctas : 2;
    if (t.subtract_fft != 0 && t.subtract_fft != 1) return snprintf(err, errlen, "subtract_fft must be 0 or 1"), false;
    g.subfft = t.subtract_fft;
    if (t.pcg_cluster != 0 && t.pcg_cluster != 8 && t.pcg_cluster != 16)
        return snprintf(err, errlen, "pcg_cluster must be 0, 8 or 16"), false;
    g.pcg_cluster = t.pcg_cluster;
    return true;
}

double time_fit(sfft_plan_t p, const void *sci, const void *tmpl, const uint8_t *mask, double *coeffs, void *diff,
                int trials) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.0;
    }
    double best = -1.0;
    // one untimed run, then the best of `trials`
    for (int t = -1; t < trials; t++) {
        cudaEventRecord(a, p->stream);
        if (sfft_fit(p, sci, tmpl, mask, nullptr, coeffs, nullptr) != SFFT_OK) break;
        if (sfft_subtract(p, sci, tmpl, coeffs, diff) != SFFT_OK) break;
        cudaEventRecord(b, p->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (t >= 0 && (best < 0 || ms < best)) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (sfft_sync_status(p) != SFFT_OK) return -1.0;
    return best;
}

}  // namespace

namespace sfft {

bool plan_geometry(const sfft_desc &d, Geometry &g, char *err, size_t errlen) {
    if (!make_geometry(d, g, err, errlen)) return false;
    sfft_tuning t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key_of(d));
        if (it == g_tune.end()) return true;
        t = it->second;
    }
    return apply_tuning(t, g, err, errlen);
}

}  // namespace sfft

// ---------------------------------------------------------------------------------------
// batch executor

struct sfft_batch_s {
    sfft_desc base{};
    std::vector<sfft_pair> pairs;
    int lanes = 1;
    bool graph = false;
    cudaStream_t user = nullptr, origin = nullptr;
    std::vector<cudaStream_t> ls;
    std::vector<std::vector<int>> lane_pairs;      // pair indices per lane, in order
    std::vector<sfft_plan_t> plan_of;              // plan of each pair
    std::vector<sfft_plan_t> plans;                // owned
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    std::vector<cudaEvent_t> ev_in;  // per lane: its first pair's host inputs are on the device
    double *rec = nullptr;                         // per pair: [status, flag0 flag1, flag2, scal0, scal1, scal2, -, -]
    sfft_cnn_t cnn = nullptr;                      // warm-start network (nullable)
    std::vector<int> stamp_row;                    // per pair: its row of stamps_buf / x0_buf, -1: none
    int nstamped = 0, n_unk = 0;
    float *stamps_buf = nullptr;                   // [nstamped][18][32][32] gathered stamps
    double *x0_buf = nullptr;                      // [nstamped][n_unk] the network's warm starts
    cudaGraph_t graph_h = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;
};

namespace {

constexpr int kRec = 8;

// ny rows of `width` bytes, `pitch` bytes apart on both sides: one contiguous copy when the
// rows touch (a 2-D copy of narrow rows, such as a mask's, runs far below the link's rate)
cudaError_t copy_frame(void *dst, const void *src, size_t pitch, size_t width, int ny, cudaMemcpyKind kind,
                       cudaStream_t s) {
    if (pitch == width) return cudaMemcpyAsync(dst, src, width * (size_t)ny, kind, s);
    return cudaMemcpy2DAsync(dst, pitch, src, pitch, width, ny, kind, s);
}

constexpr size_t kStampFloats = 18 * 32 * 32;

// queue the whole batch: the warm starts of the stamped pairs (network on the origin
// stream), fork from `origin` into the lanes, run each lane's pairs, join
cudaError_t queue_batch(sfft_batch_t b, sfft_status *st) {
    cudaError_t e = cudaSuccess;
    if (b->cnn && b->nstamped > 0) {
        for (size_t i = 0; i < b->pairs.size() && e == cudaSuccess; i++)
            if (b->stamp_row[i] >= 0)
                e = cudaMemcpyAsync(b->stamps_buf + (size_t)b->stamp_row[i] * kStampFloats, b->pairs[i].psf_stamps,
                                    kStampFloats * sizeof(float), cudaMemcpyDeviceToDevice, b->origin);
        const cudaStream_t prev = cnn_stream(b->cnn);
        sfft_cnn_set_stream(b->cnn, reinterpret_cast<sfft_stream_t>(b->origin));
        const int mb = cnn_max_batch(b->cnn);
        for (int r0 = 0; r0 < b->nstamped && e == cudaSuccess; r0 += mb) {
            const int cnt = std::min(mb, b->nstamped - r0);
            sfft_status s = sfft_cnn_warm_start(b->cnn, b->stamps_buf + (size_t)r0 * kStampFloats, cnt, b->n_unk,
                                                b->x0_buf + (size_t)r0 * b->n_unk);
            if (s != SFFT_OK) {
                *st = s;
                e = cudaErrorUnknown;
            }
        }
        sfft_cnn_set_stream(b->cnn, reinterpret_cast<sfft_stream_t>(prev));
        if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(b->ev_fork, b->origin);
    int prev_in = -1;  // last lane whose first pair copied host inputs
    for (int l = 0; l < b->lanes && e == cudaSuccess; l++) {
        e = cudaStreamWaitEvent(b->ls[l], b->ev_fork, 0);
        bool first = true;
        for (int pi : b->lane_pairs[l]) {
            if (e != cudaSuccess) break;
            const sfft_pair &q = b->pairs[pi];
            sfft_plan_t p = b->plan_of[pi];
            const size_t elt = b->base.dtype == SFFT_F64 ? 8 : 4;
            const size_t pitch = q.pitch ? q.pitch : q.nx;
            if (q.sci_host) {  // this pair's inputs, on its own lane
                // the lanes' first input copies go one after another, so that the first lane
                // starts computing after one pair's transfer instead of after all of them
                if (first && prev_in >= 0) e = cudaStreamWaitEvent(b->ls[l], b->ev_in[prev_in], 0);
                if (e == cudaSuccess)
                    e = copy_frame(const_cast<void *>(q.sci), q.sci_host, pitch * elt, q.nx * elt, q.ny,
                               cudaMemcpyHostToDevice, b->ls[l]);
                if (e == cudaSuccess && q.tmpl_host)
                    e = copy_frame(const_cast<void *>(q.tmpl), q.tmpl_host, pitch * elt, q.nx * elt, q.ny,
                                   cudaMemcpyHostToDevice, b->ls[l]);
                if (e == cudaSuccess && q.mask && q.mask_host)
                    e = copy_frame(const_cast<uint8_t *>(q.mask), q.mask_host, pitch, q.nx, q.ny, cudaMemcpyHostToDevice,
                                   b->ls[l]);
                if (e == cudaSuccess && first) {
                    e = cudaEventRecord(b->ev_in[l], b->ls[l]);
                    prev_in = l;
                }
                if (e != cudaSuccess) break;
            }
            first = false;
            const double *x0 = b->stamp_row[pi] >= 0 ? b->x0_buf + (size_t)b->stamp_row[pi] * b->n_unk : q.x0;
            sfft_status s = sfft_fit(p, q.sci, q.tmpl, q.mask, x0, q.coeffs, nullptr);
            if (s == SFFT_OK) s = sfft_subtract(p, q.sci, q.tmpl, q.coeffs, q.diff);
            if (s != SFFT_OK) {
                *st = s;
                e = cudaErrorUnknown;
                break;
            }
            if (q.coeffs_host)
                e = cudaMemcpyAsync(q.coeffs_host, q.coeffs, sizeof(double) * p->g.n, cudaMemcpyDeviceToHost, b->ls[l]);
            if (e == cudaSuccess && q.diff_host)
                e = copy_frame(q.diff_host, q.diff, pitch * elt, q.nx * elt, q.ny, cudaMemcpyDeviceToHost, b->ls[l]);
            if (e != cudaSuccess) break;
            // the pair's outcome: status word, solver flags and norms into its record
            double *r = b->rec + (size_t)pi * kRec;
            e = cudaMemcpyAsync(r, p->ws.status, sizeof(int), cudaMemcpyDeviceToDevice, b->ls[l]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r + 1, p->ws.flags, 3 * sizeof(int), cudaMemcpyDeviceToDevice, b->ls[l]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r + 3, p->ws.scal, 3 * sizeof(double), cudaMemcpyDeviceToDevice, b->ls[l]);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->ws.status, 0, sizeof(int), b->ls[l]);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[l], b->ls[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_join[l], 0);
    }
    return e;
}

void free_batch(sfft_batch_t b) {
    if (!b) return;
    if (b->origin) cudaStreamSynchronize(b->origin);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph_h) cudaGraphDestroy(b->graph_h);
    for (sfft_plan_t p : b->plans) sfft_destroy(p);
    for (cudaStream_t s : b->ls)
        if (s) cudaStreamDestroy(s);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (cudaEvent_t ev : b->ev_join)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : b->ev_in)
        if (ev) cudaEventDestroy(ev);
    if (b->rec) cudaFree(b->rec);
    if (b->stamps_buf) cudaFree(b->stamps_buf);
    if (b->x0_buf) cudaFree(b->x0_buf);
    delete b;
}

}  // namespace

extern "C" {

sfft_status sfft_tuning_get(const sfft_desc *desc, sfft_tuning *t, int32_t *cached) {
    if (!desc || !t) return set_global_error("sfft_tuning_get: null argument"), SFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(*desc));
    memset(t, 0, sizeof *t);
    if (it != g_tune.end()) *t = it->second;
    if (cached) *cached = it != g_tune.end();
    return SFFT_OK;
}

sfft_status sfft_tuning_set(const sfft_desc *desc, const sfft_tuning *t) {
    if (!desc || !t) return set_global_error("sfft_tuning_set: null argument"), SFFT_ERR_INVALID_ARG;
    Geometry g;
    char err[256];
    if (!make_geometry(*desc, g, err, sizeof err) || !apply_tuning(*t, g, err, sizeof err)) {
        errf("sfft_tuning_set: %s", err);
        return SFFT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key_of(*desc)] = *t;
    return SFFT_OK;
}

sfft_status sfft_tuning_save(const char *path) {
    if (!path) return set_global_error("sfft_tuning_save: null path"), SFFT_ERR_INVALID_ARG;
    FILE *f = fopen(path, "w");
    if (!f) return errf("sfft_tuning_save: cannot open %s", path), SFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "# ny nx pitch L dk db dtype precision solver refine : ycorr_bins ycorr_split ycorr_scalar subtract_ctas "
               "pcg_cluster ycorr_direct ycorr_sets subtract_fft\n");
    for (auto &kv : g_tune) {
        const Key &k = kv.first;
        const sfft_tuning &t = kv.second;
        fprintf(f, "%d %d %d %d %d %d %d %d %d %d : %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k),
                std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k),
                std::get<8>(k), std::get<9>(k), t.ycorr_bins, t.ycorr_split, t.ycorr_scalar, t.subtract_ctas,
                t.pcg_cluster, t.ycorr_direct, t.ycorr_sets, t.subtract_fft);
    }
    const bool ok = fclose(f) == 0;
    return ok ? SFFT_OK : (errf("sfft_tuning_save: write failed"), SFFT_ERR_INVALID_ARG);
}

sfft_status sfft_tuning_load(const char *path) {
    if (!path) return set_global_error("sfft_tuning_load: null path"), SFFT_ERR_INVALID_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return errf("sfft_tuning_load: cannot open %s", path), SFFT_ERR_INVALID_ARG;
    char line[512];
    int lineno = 0;
    sfft_status result = SFFT_OK;
    while (fgets(line, sizeof line, f)) {
        lineno++;
        if (line[0] == '#' || line[0] == '\n') continue;
        sfft_desc d;
        memset(&d, 0, sizeof d);
        sfft_tuning t;
        memset(&t, 0, sizeof t);
        int n = sscanf(line, "%d %d %d %d %d %d %d %d %d %d : %d %d %d %d %d %d %d %d", &d.ny, &d.nx, &d.pitch, &d.L,
                       &d.dk, &d.db, &d.dtype, &d.precision, &d.solver, &d.refine, &t.ycorr_bins, &t.ycorr_split,
                       &t.ycorr_scalar, &t.subtract_ctas, &t.pcg_cluster, &t.ycorr_direct, &t.ycorr_sets,
                       &t.subtract_fft);
        if (n != 18) {
            errf("sfft_tuning_load: %s:%d: expected 18 fields", path, lineno);
            result = SFFT_ERR_INVALID_ARG;
            break;
        }
        if ((result = sfft_tuning_set(&d, &t)) != SFFT_OK) break;
    }
    fclose(f);
    return result;
}

sfft_status sfft_autotune(const sfft_desc *desc, const void *sci, const void *tmpl, const uint8_t *mask,
                          int32_t trials, sfft_tuning *best, double *best_ms) {
    if (!desc || !sci || !tmpl) return set_global_error("sfft_autotune: null argument"), SFFT_ERR_INVALID_ARG;
    Geometry g0;
    char err[256];
    if (!make_geometry(*desc, g0, err, sizeof err)) return errf("sfft_autotune: %s", err), SFFT_ERR_INVALID_ARG;
    if (trials < 1) trials = 3;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return errf("sfft_autotune: %s", cudaGetErrorString(e)), SFFT_ERR_CUDA;
    const size_t elt = desc->dtype == SFFT_F64 ? 8 : 4;
    const size_t pitch = desc->pitch ? desc->pitch : desc->nx;
    double *coeffs = nullptr;
    void *diff = nullptr;
    e = cudaMalloc(&coeffs, sizeof(double) * g0.n);
    if (e == cudaSuccess) e = cudaMalloc(&diff, elt * pitch * desc->ny);
    if (e != cudaSuccess) {
        cudaFree(coeffs);
        cudaStreamDestroy(st);
        return errf("sfft_autotune: %s", cudaGetErrorString(e)), SFFT_ERR_OOM;
    }
    // the descriptor's current entry is replaced while candidates are timed
    sfft_tuning saved;
    int32_t had = 0;
    sfft_tuning_get(desc, &saved, &had);
    auto eval = [&](const sfft_tuning &t) -> double {
        if (sfft_tuning_set(desc, &t) != SFFT_OK) return -1.0;
        sfft_plan_t p = nullptr;
        if (sfft_plan(&p, desc, reinterpret_cast<sfft_stream_t>(st)) != SFFT_OK) return -1.0;
        double ms = time_fit(p, sci, tmpl, mask, coeffs, diff, trials);
        sfft_destroy(p);
        return ms;
    };
    sfft_tuning cur;
    memset(&cur, 0, sizeof cur);
    double cur_ms = eval(cur);
    sfft_status result = cur_ms < 0 ? SFFT_ERR_CUDA : SFFT_OK;
    // coordinate descent: the y-correlation route and kernel (the y-FFT route, measured above,
    // against the direct route's kernels and frequencies per CTA), then its split, then the
    // subtract grid
    std::vector<std::vector<sfft_tuning>> rounds;
    {
        std::vector<sfft_tuning> r;
        for (int scalar = 0; scalar <= 1; scalar++)
            for (int kg : {g0.kg_max, std::max(1, g0.kg_max / 2), std::max(1, (3 * g0.kg_max) / 4)}) {
                sfft_tuning t = cur;
                t.ycorr_direct = 1;
                t.ycorr_scalar = scalar;
                t.ycorr_bins = kg;
                r.push_back(t);
            }
        sfft_tuning one_set = cur;  // the y-FFT route with one producer set
        one_set.ycorr_sets = 1;
        r.push_back(one_set);
        rounds.push_back(r);
    }
    for (int rd = 0; rd < 3 && result == SFFT_OK; rd++) {
        std::vector<sfft_tuning> cand;
        if (rd == 0) {
            if (g0.yfft) cand = rounds[0];  // (a basis too large for the y-FFT kernels is direct already)
            else
                for (const sfft_tuning &t : rounds[0])
                    if (t.ycorr_direct && (t.ycorr_scalar == 1 || t.ycorr_bins != g0.kg_max)) cand.push_back(t);
        } else if (rd == 1) {
            Geometry g = g0;
            apply_tuning(cur, g, err, sizeof err);
            const int ys = g.yfft ? g.y2split : g.ysplit;
            const int max_ys = g.yfft ? 64 : std::max(1, g.ny / (2 * g.ytile));
            for (int v : {std::max(1, ys / 2), std::min(max_ys, 2 * ys), std::min(max_ys, ys + ys / 2)}) {
                if (v == ys) continue;
                sfft_tuning t = cur;
                t.ycorr_split = v;
                cand.push_back(t);
            }
        } else {
            for (int v : {1, 3, 4}) {
                sfft_tuning t = cur;
                t.subtract_ctas = v;
                cand.push_back(t);
            }
            if (desc->precision != SFFT_PREC_FP64 && g0.dk <= 2 && g0.h >= 1 && g0.h <= 7 && g0.db <= 4) {
                sfft_tuning t = cur;  // the FFT route of the difference image
                t.subtract_fft = 1;
                cand.push_back(t);
            }
        }
        for (const sfft_tuning &t : cand) {
            double ms = eval(t);
            if (ms > 0 && ms < cur_ms) cur_ms = ms, cur = t;
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(coeffs);
    cudaFree(diff);
    cudaStreamDestroy(st);
    if (result != SFFT_OK) {
        if (had)
            sfft_tuning_set(desc, &saved);
        else {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune.erase(key_of(*desc));
        }
        errf("sfft_autotune: the default shape failed to run");
        return result;
    }
    sfft_tuning_set(desc, &cur);
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return SFFT_OK;
}

sfft_status sfft_batch_create(sfft_batch_t *out, const sfft_desc *base, const sfft_pair *pairs, int32_t npairs,
                              int32_t lanes, int32_t flags, sfft_cnn_t cnn, sfft_stream_t stream) {
    if (!out) return set_global_error("sfft_batch_create: null output"), SFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!base || !pairs || npairs < 1) return set_global_error("sfft_batch_create: empty batch"), SFFT_ERR_INVALID_ARG;
    if (flags & ~(SFFT_BATCH_GRAPH | SFFT_BATCH_AUTOTUNE))
        return set_global_error("sfft_batch_create: unknown flags"), SFFT_ERR_INVALID_ARG;
    for (int i = 0; i < npairs; i++) {
        const sfft_pair &q = pairs[i];
        if (!q.sci || !q.tmpl || !q.coeffs || !q.diff) {
            errf("sfft_batch_create: pair %d has a null pointer", i);
            return SFFT_ERR_INVALID_ARG;
        }
    }
    Geometry g0;
    char gerr[256];
    if (!make_geometry(*base, g0, gerr, sizeof gerr)) {
        errf("sfft_batch_create: %s", gerr);
        return SFFT_ERR_INVALID_ARG;
    }
    if (cnn && cnn_n_out(cnn) != g0.nker) {
        errf("sfft_batch_create: the network has %d outputs, the basis %d kernel coefficients", cnn_n_out(cnn), g0.nker);
        return SFFT_ERR_INVALID_ARG;
    }
    sfft_batch_t b = new sfft_batch_s;
    b->base = *base;
    b->pairs.assign(pairs, pairs + npairs);
    b->cnn = cnn;
    b->n_unk = g0.n;
    b->stamp_row.assign(npairs, -1);
    if (cnn)
        for (int i = 0; i < npairs; i++)
            if (pairs[i].psf_stamps) b->stamp_row[i] = b->nstamped++;
    b->lanes = std::max(1, std::min(lanes > 0 ? lanes : 4, npairs));
    b->graph = (flags & SFFT_BATCH_GRAPH) != 0;
    b->user = reinterpret_cast<cudaStream_t>(stream);
    auto desc_of = [&](const sfft_pair &q) {
        sfft_desc d = *base;
        d.ny = q.ny;
        d.nx = q.nx;
        d.pitch = q.pitch;
        return d;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    b->ls.assign(b->lanes, nullptr);
    b->ev_join.assign(b->lanes, nullptr);
    b->ev_in.assign(b->lanes, nullptr);
    for (int l = 0; l < b->lanes && e == cudaSuccess; l++) {
        e = cudaStreamCreateWithFlags(&b->ls[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[l], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->rec, sizeof(double) * kRec * npairs);
    if (e == cudaSuccess && b->nstamped > 0) e = cudaMalloc(&b->stamps_buf, sizeof(float) * kStampFloats * b->nstamped);
    if (e == cudaSuccess && b->nstamped > 0) e = cudaMalloc(&b->x0_buf, sizeof(double) * b->n_unk * b->nstamped);
    if (e == cudaSuccess) e = cudaMemset(b->rec, 0, sizeof(double) * kRec * npairs);
    if (e != cudaSuccess) {
        errf("sfft_batch_create: %s", cudaGetErrorString(e));
        free_batch(b);
        return SFFT_ERR_CUDA;
    }
    // autotune each distinct geometry on its first pair's data
    if (flags & SFFT_BATCH_AUTOTUNE) {
        std::map<Key, int> seen;
        for (int i = 0; i < npairs; i++) {
            sfft_desc d = desc_of(pairs[i]);
            if (seen.count(key_of(d))) continue;
            seen[key_of(d)] = i;
            int32_t cached = 0;
            sfft_tuning t;
            sfft_tuning_get(&d, &t, &cached);
            if (cached) continue;
            sfft_status s = sfft_autotune(&d, pairs[i].sci, pairs[i].tmpl, pairs[i].mask, 2, nullptr, nullptr);
            if (s != SFFT_OK) {
                free_batch(b);
                return s;
            }
        }
    }
    // longest processing time first: cost ~ pixels + a fixed cost for the solve
    std::vector<int> order(npairs);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int i) { return (double)pairs[i].ny * pairs[i].nx + 4.0e6; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
    std::vector<double> load(b->lanes, 0.0);
    b->lane_pairs.assign(b->lanes, {});
    for (int i : order) {
        int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost(i);
        b->lane_pairs[l].push_back(i);
    }
    // one plan per (lane, geometry)
    b->plan_of.assign(npairs, nullptr);
    for (int l = 0; l < b->lanes; l++) {
        std::map<Key, sfft_plan_t> mine;
        for (int i : b->lane_pairs[l]) {
            sfft_desc d = desc_of(pairs[i]);
            auto it = mine.find(key_of(d));
            if (it == mine.end()) {
                sfft_plan_t p = nullptr;
                sfft_status s = sfft_plan(&p, &d, reinterpret_cast<sfft_stream_t>(b->ls[l]));
                if (s != SFFT_OK) {
                    errf("sfft_batch_create: plan for pair %d (%dx%d): %s", i, d.ny, d.nx, sfft_last_error(nullptr));
                    free_batch(b);
                    return s;
                }
                b->plans.push_back(p);
                it = mine.emplace(key_of(d), p).first;
            }
            b->plan_of[i] = it->second;
        }
    }
    // one eager pass, after the caller's queued work: kernel attributes and cluster
    // queries happen outside any capture
    sfft_status qs = SFFT_OK;
    e = cudaEventRecord(b->ev_fork, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_fork, 0);
    if (e == cudaSuccess) e = queue_batch(b, &qs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
    if (e != cudaSuccess || qs != SFFT_OK) {
        if (qs == SFFT_OK) errf("sfft_batch_create: first pass: %s", cudaGetErrorString(e));
        free_batch(b);
        return qs != SFFT_OK ? qs : SFFT_ERR_CUDA;
    }
    if (b->graph) {
        const uint64_t l0 = launch_count();
        e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t eq = queue_batch(b, &qs);
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(b->origin, &gr);
            if (eq != cudaSuccess) e = eq;
            b->graph_h = gr;
        }
        b->launches_per_run = launch_count() - l0;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph_h, 0);
        if (e != cudaSuccess || qs != SFFT_OK) {
            errf("sfft_batch_create: graph capture: %s", qs != SFFT_OK ? sfft_last_error(nullptr) : cudaGetErrorString(e));
            free_batch(b);
            return qs != SFFT_OK ? qs : SFFT_ERR_CUDA;
        }
    }
    *out = b;
    return SFFT_OK;
}

sfft_status sfft_batch_run(sfft_batch_t b) {
    if (!b) return set_global_error("sfft_batch_run: null batch"), SFFT_ERR_INVALID_ARG;
    cudaError_t e;
    sfft_status qs = SFFT_OK;
    if (b->graph) {
        e = cudaGraphLaunch(b->exec, b->user);
        if (e == cudaSuccess) note_launch((int)b->launches_per_run);
    } else {
        // order the origin stream after the caller's work, run, and make the caller wait
        cudaEvent_t ev = b->ev_fork;
        e = cudaEventRecord(ev, b->user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, ev, 0);
        if (e == cudaSuccess) e = queue_batch(b, &qs);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[0], b->origin);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev_join[0], 0);
    }
    if (qs != SFFT_OK) return qs;
    if (e != cudaSuccess) return errf("sfft_batch_run: %s", cudaGetErrorString(e)), SFFT_ERR_CUDA;
    return SFFT_OK;
}

sfft_status sfft_batch_info(sfft_batch_t b, sfft_fit_info *infos) {
    if (!b || !infos) return set_global_error("sfft_batch_info: null argument"), SFFT_ERR_INVALID_ARG;
    const int np = (int)b->pairs.size();
    std::vector<double> rec((size_t)kRec * np);
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e == cudaSuccess) e = cudaMemcpy(rec.data(), b->rec, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return errf("sfft_batch_info: %s", cudaGetErrorString(e)), SFFT_ERR_CUDA;
    const bool fast = b->base.solver == SFFT_SOLVE_PCG;
    sfft_status worst = SFFT_OK;
    for (int i = 0; i < np; i++) {
        const double *r = rec.data() + (size_t)i * kRec;
        int st, fl[3];
        memcpy(&st, r, sizeof st);
        memcpy(fl, r + 1, sizeof fl);
        sfft_fit_info &f = infos[i];
        memset(&f, 0, sizeof f);
        f.status = st;
        f.n = b->plan_of[i]->g.n;
        f.iterations = fast && fl[0] ? fl[1] : 1;
        f.fallback = fast && !fl[0] ? 1 : 0;
        f.rel_residual = r[4] > 0 ? sqrt(r[3] / r[4]) : 0.0;
        f.start_residual = fast && fl[0] && r[4] > 0 ? sqrt(r[5] / r[4]) : 1.0;
        f.pcg_status = fast && !fl[0] ? (fl[2] ? fl[2] : (int)SFFT_ERR_NOT_SPD) : 0;
        if (st != 0 && worst == SFFT_OK) worst = (sfft_status)st;
    }
    return worst;
}

void sfft_batch_destroy(sfft_batch_t b) { free_batch(b); }

sfft_status sfft_batch(const sfft_desc *base, int32_t n_sci, int32_t n_tmpl, const sfft_pair *pairs, sfft_cnn_t cnn,
                       sfft_fit_info *infos, sfft_stream_t stream) {
    if (!base || n_sci < 1 || n_tmpl < 1 || !pairs) return set_global_error("sfft_batch: empty batch"), SFFT_ERR_INVALID_ARG;
    sfft_batch_t b = nullptr;
    sfft_status s = sfft_batch_create(&b, base, pairs, n_sci * n_tmpl, 0, 0, cnn, stream);
    if (s != SFFT_OK) return s;
    // the creation pass already ran every pair once; its records are current
    if (infos) {
        s = sfft_batch_info(b, infos);
        if (s == SFFT_ERR_NOT_SPD) s = SFFT_OK;  // reported per pair
    }
    sfft_batch_destroy(b);
    return s;
}

}  // extern "C"
