// C ABI of libsfft: descriptor validation, plan geometry, workspace, twiddle tables and
// the call sequences of sfft_normal / sfft_fit / sfft_subtract / sfft_batch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "sfft_internal.cuh"

namespace {

thread_local char g_last_error[512] = "";

void set_err(sfft_plan_t p, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    snprintf(g_last_error, sizeof g_last_error, "%s", buf);
    if (p) snprintf(p->err, sizeof p->err, "%s", buf);
}

sfft_status cuda_fail(sfft_plan_t p, cudaError_t e, const char *where) {
    set_err(p, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SFFT_ERR_OOM : SFFT_ERR_CUDA;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

namespace sfft {

void set_global_error(const char *msg) { set_err(nullptr, "%s", msg); }
void default_y2split(Geometry &g);
void finish_geometry(Geometry &g);
int device_sm_count();

int default_ysplit(const Geometry &g) {
    // row chunks so the grid covers several waves of 2 CTAs on each of 152 SMs
    const int units = g.nseg * ((g.nkf + g.kg - 1) / g.kg);
    int ys = (4 * 304 + units - 1) / units;
    const int max_ys = g.ny / (2 * g.ytile);
    if (ys > max_ys) ys = max_ys;
    return ys < 1 ? 1 : ys;
}

bool make_geometry(const sfft_desc &d, Geometry &g, char *err, size_t errlen) {
    memset(&g, 0, sizeof g);
    g.sub_per_sm = 2;
    if (d.ny < 1 || d.nx < 1) return snprintf(err, errlen, "ny, nx must be >= 1"), false;
    if (d.L < 1 || d.L % 2 == 0) return snprintf(err, errlen, "L must be odd and >= 1 (got %d)", d.L), false;
    if (d.ny < d.L || d.nx < d.L) return snprintf(err, errlen, "frame %dx%d smaller than L=%d", d.ny, d.nx, d.L), false;
    if (d.dk < 0 || d.db < 0) return snprintf(err, errlen, "dk, db must be >= 0"), false;
    if (d.dtype != SFFT_F32 && d.dtype != SFFT_F64) return snprintf(err, errlen, "unknown dtype %d", d.dtype), false;
    if (d.precision != SFFT_PREC_FP32 && d.precision != SFFT_PREC_SPLIT && d.precision != SFFT_PREC_FP64)
        return snprintf(err, errlen, "unknown precision %d", d.precision), false;
    if (d.solver != SFFT_SOLVE_CHOLESKY && d.solver != SFFT_SOLVE_PCG)
        return snprintf(err, errlen, "unknown solver %d", d.solver), false;
    g.pitch = d.pitch ? d.pitch : d.nx;
    if (g.pitch < d.nx) return snprintf(err, errlen, "pitch %d < nx %d", g.pitch, d.nx), false;
    g.ny = d.ny;
    g.nx = d.nx;
    g.L = d.L;
    g.h = (d.L - 1) / 2;
    g.dk = d.dk;
    g.db = d.db;
    g.nk = npoly(d.dk);
    g.nb = npoly(d.db);
    g.nker = g.nk * d.L * d.L;
    g.n = g.nker + g.nb;
    g.P = d.seg ? d.seg : 256;
    if (g.P != 256) return snprintf(err, errlen, "segment FFT length %d not supported (256 only)", g.P), false;
    g.G = d.L - 1;
    g.U = g.P - 2 * g.G;
    if (g.U < 1) return snprintf(err, errlen, "L=%d too large for segment length %d", d.L, g.P), false;
    g.nseg = (d.nx + g.U - 1) / g.U;
    g.nkf = g.P / 2 + 1;
    g.nimg = 2 * g.nk + g.nb + 1;
    g.nimg_pad = (g.nimg + 1) & ~1;
    if (g.nimg_pad > 32) return snprintf(err, errlen, "dk=%d, db=%d give %d images per segment (max 32)", d.dk, d.db, g.nimg), false;
    g.npair = g.nk * (g.nk + 1) / 2;
    g.nent = g.npair * (2 * d.L - 1) + g.nk * (g.nb + 1) * d.L;
    g.C = d.L;
    if (g.C > 15) return snprintf(err, errlen, "L=%d > 15 not supported", d.L), false;
    g.items_per_k = 2 * g.npair + g.nk * (g.nb + 1);
    if (g.items_per_k > 256) return snprintf(err, errlen, "dk=%d, db=%d need %d work items per frequency (max 256)", d.dk, d.db, g.items_per_k), false;
    g.ytile = 64;
    {
        // frequencies per CTA: as many items as fit 256 threads, and two double-buffered
        // tiles within the shared-memory budget (two CTAs per SM for FP32 spectra)
        const size_t cpx_sz = d.precision == SFFT_PREC_FP64 ? 16 : 8;
        const size_t per_k = 2 * (size_t)(g.ytile + 2 * g.G) * g.nimg_pad * cpx_sz;
        const size_t per_k_ws = 2 * (size_t)(g.ytile + 2 * g.G) * (((g.nk + 1) & ~1) + 2) * cpx_sz;
        const size_t budget = d.precision == SFFT_PREC_FP64 ? 200 * 1024 : 112 * 1024;
        auto pick = [&](int items, size_t pk) {
            int kg = 256 / items;
            int kg_smem = (int)(budget / pk);
            if (kg > kg_smem) kg = kg_smem;
            if (kg > g.nkf) kg = g.nkf;
            return kg < 1 ? 1 : kg;
        };
        g.kg = pick(g.items_per_k, per_k);
        g.kg_max = g.kg;
        g.kg_ws = pick(g.nk, per_k_ws);
        if (per_k > budget) return snprintf(err, errlen, "y-correlation tile does not fit shared memory"), false;
        g.ysplit = default_ysplit(g);
        // refinement pass: one thread per (segment, chunk, frequency, W_i); ~200k threads
        long per_chunk = (long)g.nseg * g.nkf * g.nk;
        int yc = (int)((200000 + per_chunk - 1) / per_chunk);
        int max_yc = d.ny / 32;
        if (yc > max_yc) yc = max_yc;
        g.ychunks_ws = yc < 1 ? 1 : yc;
    }
    g.refine = d.refine < 0 ? 0 : (d.refine > 0 ? d.refine : (d.precision == SFFT_PREC_SPLIT ? 1 : 0));
    if (d.db > 4) return snprintf(err, errlen, "db=%d > 4 not supported", d.db), false;
    {
        // moments CTAs of 128 rows when that still gives 1.5 CTAs per SM, else 64 rows (at most
        // the moments kernel's 128): fewer, fuller CTAs halve the per-CTA FP64 epilogue
        const long ctas128 = (long)((g.nx + 511) / 512) * ((g.ny + 127) / 128);
        g.mom_rows = 2 * ctas128 >= 3L * device_sm_count() ? 128 : 64;
    }
    g.mom_ctas = moments_ctas(g);
    g.nmom = npoly(2 * d.db) + npoly(d.db);
    g.pmax = d.dk > 2 * d.db ? d.dk : 2 * d.db;
    if (d.spin_limit < 0) return snprintf(err, errlen, "spin_limit must be >= 0"), false;
    g.spin_limit = d.spin_limit > 0 ? (long long)d.spin_limit : (1ll << 24);
    // y-block FFT route (the default): blocks of Py = 128 rows, Uy = Py - 2G of them new
    g.nbase = 2 * (d.dk + 1) + (d.db + 1) + 1;
    g.Py = 128;
    g.Uy = g.Py - 2 * g.G;
    g.nyb = (d.ny + g.Uy - 1) / g.Uy;
    g.npair_all = g.npair + g.nk * (g.nb + 1);
    g.yfft = 1;
    {
        // pairs per CTA: at most 64 (16 per thread, 4 threads per ky in the FP32 layout) and
        // what the shared-memory budget leaves; groups balanced
        int ypg = g.npair_all < 64 ? g.npair_all : 64;
        for (;;) {
            g.ypg = ypg;
            if (ypg == 1 || yfft_smem_bytes(g, d.precision, false) <= (size_t)220 * 1024) break;
            ypg--;
        }
        g.npg = (g.npair_all + ypg - 1) / ypg;
        g.ypg = (g.npair_all + g.npg - 1) / g.npg;
        if (yfft_smem_bytes(g, d.precision, false) > (size_t)220 * 1024 ||
            yfft_smem_bytes(g, d.precision, true) > (size_t)220 * 1024)
            g.yfft = 0;  // this basis is too large for the y-FFT kernels: the direct route runs it
    }
    default_y2split(g);
    g.ysets = 2;
    g.subfft = 0;
    finish_geometry(g);
    return true;
}

// CTAs per frequency of the y-FFT kernels: the main pass runs one 512-thread CTA per SM, so
// its split is the one (at least 8 units per CTA) whose last wave is fullest; the
// refinement pass (256 threads, several CTAs per SM) takes about four CTAs per SM
void default_y2split(Geometry &g) {
    const int sms = device_sm_count();
    const int units = g.nseg * g.nyb;
    int best = 1;
    double best_eff = -1.0;
    for (int sp = 1; sp <= 16; sp++) {
        if (sp > 1 && units / sp < 8) break;
        const long ctas = (long)g.nkf * sp * g.npg;
        const long waves = (ctas + sms - 1) / sms;
        const double eff = (double)ctas / (double)(waves * sms);
        if (eff > best_eff + 1e-9) best_eff = eff, best = sp;
    }
    g.y2split = best;
    int ws = (4 * sms + g.nkf - 1) / g.nkf;
    if (ws > units) ws = units;
    g.y2split_ws = ws < 1 ? 1 : (ws > 16 ? 16 : ws);
}

// fields that follow from the route: values per spectrum record
void finish_geometry(Geometry &g) { g.nrec = g.yfft ? (g.nbase + 1) & ~1 : g.nimg_pad; }

int device_sm_count() {
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v > 0) return v;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return 152;  // no device visible (host-only calls): the GB300's count
    }
    cached.store(sms);
    return sms;
}

struct Carve {
    size_t off = 0;
    template <class T>
    T *take(void *base, size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(static_cast<char *>(base) + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

static size_t carve(const Geometry &g, int precision, int dtype, void *base, Workspace *w) {
    Carve c;
    const size_t dtype_size = dtype == SFFT_F64 ? 8 : 4;
    const size_t cpx_sz = precision == SFFT_PREC_FP64 ? 16 : 8;
    Workspace tmp;
    Workspace &o = w ? *w : tmp;
    o.spec = c.take<char>(base, (size_t)g.nseg * g.nkf * g.ny * g.nrec * cpx_sz);
    {
        // K2 partial sums, 16 bytes per complex value: y-FFT route [split][nkf][pairs][Py];
        // direct route [segment][chunk][nkf][entry], or (refinement) the W x S_m partials
        size_t main_v, ws_v;
        if (g.yfft) {
            main_v = (size_t)g.y2split * g.nkf * g.npair_all * g.Py;
            const size_t ws_fft = (size_t)g.y2split_ws * g.nkf * g.nk * g.Py;
            const size_t ws_dir = (size_t)g.nseg * g.ychunks_ws * g.nkf * g.nk * g.L;
            ws_v = ws_fft > ws_dir ? ws_fft : ws_dir;
        } else {
            main_v = (size_t)g.nseg * g.ysplit * g.nkf * g.nent;
            ws_v = (size_t)g.nseg * g.ychunks_ws * g.nkf * g.nk * g.L;
        }
        o.ypart = c.take<double>(base, 2 * (main_v > ws_v ? main_v : ws_v));
    }
    o.resid = g.refine ? c.take<char>(base, (size_t)g.ny * g.pitch * (dtype_size)) : nullptr;
    o.rspec = g.refine && (precision != SFFT_PREC_FP64 || g.yfft)
                  ? c.take<char>(base, (size_t)g.nseg * g.ny * g.nkf * cpx_sz) : nullptr;
    o.ysum = c.take<double>(base, (size_t)g.nkf * g.nent * 2);
    o.lagww = c.take<double>(base, (size_t)g.npair * (2 * g.L - 1) * (2 * g.L - 1));
    o.lagwg = c.take<double>(base, (size_t)g.nk * g.nb * g.L * g.L);
    o.lagws = c.take<double>(base, (size_t)g.nk * g.L * g.L);
    {
        // moment partials: of the moments kernel, or of the FP32 refinement's residual kernel
        const size_t a = (size_t)g.mom_ctas * g.nmom, r = (size_t)residual_ctas_max(g) * g.nb;
        o.mom_part = c.take<double>(base, a > r ? a : r);
    }
    o.mom = c.take<double>(base, (size_t)g.nmom);
    o.N = c.take<double>(base, (size_t)g.n * g.n);
    o.b = c.take<double>(base, (size_t)g.n);
    o.R = c.take<double>(base, (size_t)g.n * g.n);
    o.x = c.take<double>(base, (size_t)g.n);
    o.r = c.take<double>(base, (size_t)g.n);
    o.z = c.take<double>(base, (size_t)g.n);
    o.p = c.take<double>(base, (size_t)g.n);
    o.q = c.take<double>(base, (size_t)g.n);
    o.b2 = c.take<double>(base, (size_t)g.n);
    o.scal = c.take<double>(base, 16);
    o.dinv = c.take<double>(base, (size_t)g.n);
    o.Rf = c.take<float>(base, (size_t)g.n * g.n);
    o.dscale = c.take<double>(base, (size_t)g.n);
    o.Lg = c.take<float>(base, pcg_factor_floats(g));
    o.flags = c.take<int>(base, 16);
    o.dinvf = c.take<float>(base, (size_t)g.n);
    o.cfold = c.take<char>(base, (size_t)g.ny * g.L * (g.dk + 1) * g.L * (cpx_sz / 2) + (size_t)g.ny * (g.db + 1) * (cpx_sz / 2));
    o.kspec = c.take<float2>(base, (size_t)g.nk * g.L * 128);
    o.status = c.take<int>(base, 16);
    o.bar = c.take<unsigned>(base, 16);
    o.tw_fft = c.take<char>(base, (size_t)2 * g.P * cpx_sz);
    o.xpow = c.take<char>(base, (size_t)(g.pmax + 1) * g.nx * (cpx_sz / 2));
    o.ypow = c.take<char>(base, (size_t)(g.pmax + 1) * g.ny * (cpx_sz / 2));
    o.tw_x = c.take<double>(base, (size_t)g.nkf * (2 * g.G + 1) * 2);
    o.tw_y = c.take<char>(base, (size_t)2 * g.Py * cpx_sz);
    o.tw_yi = c.take<char>(base, (size_t)g.Py * 16);
    return align_up(c.off, 256);
}

size_t workspace_bytes(const Geometry &g, int precision, int dtype) {
    return carve(g, precision, dtype, nullptr, nullptr);
}

static std::atomic<uint64_t> g_launches{0};
void note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Records a CUDA event pair around one stage on the plan's stream while profiling is on.
struct StageTimer {
    sfft_plan_t p;
    int stage;
    cudaEvent_t a = nullptr;
    static cudaEvent_t get(sfft_plan_t p) {
        cudaEvent_t e = nullptr;
        if (!p->ev_free.empty()) {
            e = p->ev_free.back();
            p->ev_free.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }
    StageTimer(sfft_plan_t p_, int stage_) : p(p_), stage(stage_) {
        if (p->profile && (a = get(p)) != nullptr) cudaEventRecord(a, p->stream);
    }
    ~StageTimer() {
        if (!a) return;
        cudaEvent_t b = get(p);
        if (!b) {
            p->ev_free.push_back(a);
            return;
        }
        cudaEventRecord(b, p->stream);
        p->ev_pending[stage].push_back({a, b});
    }
};

}  // namespace sfft

using namespace sfft;

extern "C" {

const char *sfft_status_string(sfft_status s) {
    switch (s) {
        case SFFT_OK: return "ok";
        case SFFT_ERR_INVALID_ARG: return "invalid argument";
        case SFFT_ERR_CUDA: return "CUDA error";
        case SFFT_ERR_OOM: return "out of memory";
        case SFFT_ERR_NOT_SPD: return "normal matrix not positive definite";
        case SFFT_ERR_NO_CONVERGENCE: return "solver did not converge";
        case SFFT_ERR_TIMEOUT: return "device wait timed out";
        case SFFT_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sfft_last_error(sfft_plan_t plan) { return plan ? plan->err : g_last_error; }

sfft_status sfft_workspace_size(const sfft_desc *desc, size_t *bytes) {
    if (!desc || !bytes) return set_err(nullptr, "null argument"), SFFT_ERR_INVALID_ARG;
    Geometry g;
    char err[256];
    if (!plan_geometry(*desc, g, err, sizeof err)) return set_err(nullptr, "%s", err), SFFT_ERR_INVALID_ARG;
    *bytes = workspace_bytes(g, desc->precision, desc->dtype);
    return SFFT_OK;
}

sfft_status sfft_plan(sfft_plan_t *plan, const sfft_desc *desc, sfft_stream_t stream) {
    if (!plan) return set_err(nullptr, "null plan pointer"), SFFT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!desc) return set_err(nullptr, "null descriptor"), SFFT_ERR_INVALID_ARG;
    Geometry g;
    char err[256];
    if (!plan_geometry(*desc, g, err, sizeof err)) {
        bool unsup = strstr(err, "not supported") || strstr(err, "not built");
        set_err(nullptr, "%s", err);
        return unsup ? SFFT_ERR_UNSUPPORTED : SFFT_ERR_INVALID_ARG;
    }
    size_t bytes = workspace_bytes(g, desc->precision, desc->dtype);
    if (desc->workspace_cap && bytes > desc->workspace_cap) {
        set_err(nullptr, "workspace %zu bytes exceeds cap %zu", bytes, desc->workspace_cap);
        return SFFT_ERR_OOM;
    }
    sfft_plan_t p = new (std::nothrow) sfft_plan_s();
    if (!p) return set_err(nullptr, "host allocation failed"), SFFT_ERR_OOM;
    p->desc = *desc;
    p->g = g;
    p->stream = reinterpret_cast<cudaStream_t>(stream);
    p->err[0] = 0;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        sfft_status s = cuda_fail(nullptr, e, "cudaGetDevice");
        delete p;
        return s;
    }
    e = cudaMalloc(&p->ws.base, bytes);
    if (e != cudaSuccess) {
        sfft_status s = cuda_fail(nullptr, e, "workspace allocation");
        delete p;
        return s;
    }
    p->ws.bytes = bytes;
    carve(g, desc->precision, desc->dtype, p->ws.base, &p->ws);

    // twiddles from FP64 trigonometry: forward FFT exp(-2 pi i m / P), and the x-direction
    // inverse-DFT weights w_k exp(+2 pi i k m / P) / P for m in [0, 2G], w_0 = w_{P/2} = 1, else 2
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<double> twx((size_t)g.nkf * (2 * g.G + 1) * 2);
    for (int k = 0; k < g.nkf; k++) {
        double wk = (k == 0 || 2 * k == g.P) ? 1.0 : 2.0;
        for (int m = 0; m <= 2 * g.G; m++) {
            long km = ((long)k * m) % g.P;
            double ang = two_pi * (double)km / g.P;
            twx[((size_t)k * (2 * g.G + 1) + m) * 2] = wk * cos(ang) / g.P;
            twx[((size_t)k * (2 * g.G + 1) + m) * 2 + 1] = wk * sin(ang) / g.P;
        }
    }
    e = cudaMemcpyAsync(p->ws.tw_x, twx.data(), twx.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    // forward FFT twiddles exp(-2 pi i m / P): high part then remainder (zero for FP64)
    std::vector<double> tw64((size_t)g.P * 4, 0.0);
    std::vector<float> tw((size_t)g.P * 4, 0.0f);
    if (e == cudaSuccess) {
        if (desc->precision == SFFT_PREC_FP64) {
            for (int m = 0; m < g.P; m++) {
                tw64[2 * m] = cos(two_pi * m / g.P);
                tw64[2 * m + 1] = -sin(two_pi * m / g.P);
            }
            e = cudaMemcpyAsync(p->ws.tw_fft, tw64.data(), tw64.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream);
        } else {
            for (int m = 0; m < g.P; m++) {
                double c = cos(two_pi * m / g.P), sn = -sin(two_pi * m / g.P);
                float ch = (float)c, sh = (float)sn;
                tw[2 * m] = ch;
                tw[2 * m + 1] = sh;
                tw[2 * (g.P + m)] = (float)(c - (double)ch);
                tw[2 * (g.P + m) + 1] = (float)(sn - (double)sh);
            }
            e = cudaMemcpyAsync(p->ws.tw_fft, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream);
        }
    }
    // coordinate power tables xh^p, yh^q (p, q <= pmax): FP64 powers rounded once
    std::vector<double> xp64((size_t)(g.pmax + 1) * g.nx), yp64((size_t)(g.pmax + 1) * g.ny);
    std::vector<float> xp32(xp64.size()), yp32(yp64.size());
    for (int axis = 0; axis < 2; axis++) {
        int len = axis ? g.ny : g.nx;
        std::vector<double> &t = axis ? yp64 : xp64;
        for (int i = 0; i < len; i++) {
            double c = len > 1 ? (2.0 * i - (len - 1)) / (double)(len - 1) : 0.0, v = 1.0;
            for (int q = 0; q <= g.pmax; q++) {
                t[(size_t)q * len + i] = v;
                v *= c;
            }
        }
    }
    for (size_t i = 0; i < xp64.size(); i++) xp32[i] = (float)xp64[i];
    for (size_t i = 0; i < yp64.size(); i++) yp32[i] = (float)yp64[i];
    if (e == cudaSuccess) {
        if (desc->precision == SFFT_PREC_FP64) {
            e = cudaMemcpyAsync(p->ws.xpow, xp64.data(), xp64.size() * 8, cudaMemcpyHostToDevice, p->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws.ypow, yp64.data(), yp64.size() * 8, cudaMemcpyHostToDevice, p->stream);
        } else {
            e = cudaMemcpyAsync(p->ws.xpow, xp32.data(), xp32.size() * 4, cudaMemcpyHostToDevice, p->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(p->ws.ypow, yp32.data(), yp32.size() * 4, cudaMemcpyHostToDevice, p->stream);
        }
    }
    // y-block FFT twiddles: forward exp(-2 pi i m / Py) (FP32: high part and remainder) and the
    // inverse exp(+2 pi i m / Py) (FP32: double-float (cos hi, sin hi, cos lo, sin lo))
    std::vector<double> twy64((size_t)g.Py * 4, 0.0), twyi64((size_t)g.Py * 2);
    std::vector<float> twy32((size_t)g.Py * 4, 0.0f), twyi32((size_t)g.Py * 4);
    for (int m = 0; m < g.Py; m++) {
        const double c = cos(two_pi * m / g.Py), sn = sin(two_pi * m / g.Py);
        twy64[2 * m] = c;
        twy64[2 * m + 1] = -sn;
        const float ch = (float)c, sh = (float)-sn;
        twy32[2 * m] = ch;
        twy32[2 * m + 1] = sh;
        twy32[2 * (g.Py + m)] = (float)(c - (double)ch);
        twy32[2 * (g.Py + m) + 1] = (float)(-sn - (double)sh);
        twyi64[2 * m] = c;
        twyi64[2 * m + 1] = sn;
        const float ih = (float)c, jh = (float)sn;
        twyi32[4 * m] = ih;
        twyi32[4 * m + 1] = jh;
        twyi32[4 * m + 2] = (float)(c - (double)ih);
        twyi32[4 * m + 3] = (float)(sn - (double)jh);
    }
    if (e == cudaSuccess) {
        const bool f64 = desc->precision == SFFT_PREC_FP64;
        e = f64 ? cudaMemcpyAsync(p->ws.tw_y, twy64.data(), twy64.size() * 8, cudaMemcpyHostToDevice, p->stream)
                : cudaMemcpyAsync(p->ws.tw_y, twy32.data(), twy32.size() * 4, cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = f64 ? cudaMemcpyAsync(p->ws.tw_yi, twyi64.data(), twyi64.size() * 8, cudaMemcpyHostToDevice, p->stream)
                    : cudaMemcpyAsync(p->ws.tw_yi, twyi32.data(), twyi32.size() * 4, cudaMemcpyHostToDevice, p->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ws.status, 0, 16 * sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // host staging vectors die here
    if (e != cudaSuccess) {
        sfft_status s = cuda_fail(nullptr, e, "plan set-up");
        cudaFree(p->ws.base);
        delete p;
        return s;
    }
    *plan = p;
    return SFFT_OK;
}

void sfft_destroy(sfft_plan_t plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    for (auto &v : plan->ev_pending)
        for (auto &pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : plan->ev_free) cudaEventDestroy(e);
    cudaFree(plan->ws.base);
    delete plan;
}

sfft_status sfft_profile(sfft_plan_t plan, int32_t enable) {
    if (!plan) return set_err(nullptr, "null plan"), SFFT_ERR_INVALID_ARG;
    plan->profile = enable != 0;
    return SFFT_OK;
}

sfft_status sfft_stage_times(sfft_plan_t plan, double *ms, int32_t *calls) {
    if (!plan || !ms) return set_err(plan, "null argument"), SFFT_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(plan, e, "stage-time sync");
    for (int st = 0; st < SFFT_NSTAGES; st++) {
        double sum = 0.0;
        for (auto &pr : plan->ev_pending[st]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) sum += t;
            plan->ev_free.push_back(pr.first);
            plan->ev_free.push_back(pr.second);
        }
        plan->ev_pending[st].clear();
        ms[st] = sum;
    }
    if (calls) *calls = plan->timed_calls;
    plan->timed_calls = 0;
    return SFFT_OK;
}

sfft_status sfft_launch_count(uint64_t *count) {
    if (!count) return set_err(nullptr, "null argument"), SFFT_ERR_INVALID_ARG;
    *count = g_launches.load();
    return SFFT_OK;
}

sfft_status sfft_n_unknowns(sfft_plan_t plan, int32_t *n) {
    if (!plan || !n) return set_err(plan, "null argument"), SFFT_ERR_INVALID_ARG;
    *n = plan->g.n;
    return SFFT_OK;
}

sfft_status sfft_set_stream(sfft_plan_t plan, sfft_stream_t stream) {
    if (!plan) return set_err(nullptr, "null plan"), SFFT_ERR_INVALID_ARG;
    plan->stream = reinterpret_cast<cudaStream_t>(stream);
    return SFFT_OK;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static sfft_status check_images(sfft_plan_t plan, const void *sci, const void *tmpl) {
    if (!plan) return set_err(nullptr, "null plan"), SFFT_ERR_INVALID_ARG;
    if (!sci || !tmpl) return set_err(plan, "null image pointer"), SFFT_ERR_INVALID_ARG;
    if (!aligned16(sci) || !aligned16(tmpl)) return set_err(plan, "image pointers must be 16-byte aligned"), SFFT_ERR_INVALID_ARG;
    return SFFT_OK;
}

// queue the assembly of N, b into the given device arrays
static sfft_status queue_normal(sfft_plan_t p, const void *sci, const void *tmpl, const uint8_t *mask, double *N,
                                double *b) {
    const Geometry &g = p->g;
    Workspace &w = p->ws;
    cudaStream_t st = p->stream;
    cudaError_t e;
    {
        StageTimer t(p, ST_SEGFFT);
        e = launch_segment_fft(g, p->desc.dtype, p->desc.precision, sci, tmpl, mask, w.tw_fft, w.xpow, w.ypow, w.spec, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "segment FFT launch");
    {
        StageTimer t(p, ST_MOMENTS);
        e = launch_moments(g, p->desc.dtype, p->desc.precision, sci, mask, w.ypow, w.mom_part, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "moments launch");
    {
        StageTimer t(p, ST_YCORR);
        e = g.yfft ? launch_ycorr_fft(g, p->desc.precision, w.spec, nullptr, w.ypow, w.tw_y, w.ypart, false, st)
                   : launch_ycorr(g, p->desc.precision, w.spec, w.ypart, false, nullptr, nullptr, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "y-correlation launch");
    {
        StageTimer t(p, ST_LAGS);
        if (g.yfft) e = launch_yinv(g, p->desc.precision, w.ypart, w.tw_yi, w.ysum, false, st);
        if (e == cudaSuccess)
            e = launch_lag_tables(g, w.ypart, w.ysum, w.tw_x, w.lagww, w.lagwg, w.lagws, w.mom_part, w.mom, false,
                                  p->desc.precision != SFFT_PREC_FP64, g.yfft != 0, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "lag-table launch");
    {
        StageTimer t(p, ST_ASSEMBLE);
        e = launch_assemble(g, w.lagww, w.lagwg, w.lagws, w.mom, N, b, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "assembly launch");
    return SFFT_OK;
}

// One residual refinement pass: R = S_m - sum a (w T_m)(u - d) - m sum b w (the residual of
// the fit on the masked frames), c = [Phi Psi]^T R through the same segment spectra (R gets
// its own row-segment spectra; the base spectra of the main pass are still in place), then
// theta += N^{-1} c with the existing factor.
static cudaError_t queue_refine(sfft_plan_t p, const void *sci, const void *tmpl, const uint8_t *mask,
                                double *coeffs) {
    const Geometry &g = p->g;
    Workspace &w = p->ws;
    cudaStream_t st = p->stream;
    const int slot = 2 * g.nk + g.nb;
    // the FP32 path's residual kernel also sums the residual's background moments into mom
    const bool fp32 = p->desc.precision != SFFT_PREC_FP64;
    cudaError_t e = launch_subtract(g, p->desc.dtype, p->desc.precision, sci, tmpl, mask, true, coeffs, w.xpow,
                                    w.ypow, w.cfold, w.resid, fp32 ? w.mom_part : nullptr, fp32 ? w.mom : nullptr, st);
    if (e == cudaSuccess) e = launch_segment_fft_single(g, p->desc.dtype, p->desc.precision, w.resid, w.tw_fft, slot,
                                                        w.spec, w.rspec, st);
    if (e == cudaSuccess && !fp32)
        e = launch_moments(g, p->desc.dtype, p->desc.precision, w.resid, mask, w.ypow, w.mom_part, st);
    // W_i x R: the direct row correlation on the FP32 paths (either spectrum layout), the
    // y-FFT kernels for FP64 spectra on the y-FFT route
    const bool ws_fft = g.yfft && !fp32;
    if (e == cudaSuccess)
        e = ws_fft ? launch_ycorr_fft(g, p->desc.precision, w.spec, w.rspec, w.ypow, w.tw_y, w.ypart, true, st)
                   : launch_ycorr(g, p->desc.precision, w.spec, w.ypart, true, w.rspec, w.ypow, st);
    if (e == cudaSuccess && ws_fft) e = launch_yinv(g, p->desc.precision, w.ypart, w.tw_yi, w.ysum, true, st);
    if (e == cudaSuccess)
        e = launch_lag_tables(g, w.ypart, w.ysum, w.tw_x, w.lagww, w.lagwg, w.lagws, fp32 ? nullptr : w.mom_part,
                              w.mom, true, fp32, ws_fft, st);
    if (e == cudaSuccess) e = launch_refine_rhs(g, w.lagws, w.mom, w.q, st);
    // correction x += N^{-1} c: with the cluster factor when the fast solver converged, else
    // with the FP32 copy of the FP64 Cholesky factor (each launch checks the flag)
    if (e == cudaSuccess && p->desc.solver == SFFT_SOLVE_PCG && pcg_cluster_size(g) > 0)
        e = launch_pcg_cluster(g, w.N, w.q, nullptr, coeffs, w.r, w.p, w.b2, w.z, w.dscale, w.Lg, w.scal, w.flags,
                               0, 0.0, true, st);
    if (e == cudaSuccess)
        e = launch_cholesky_solve(g, w.N, w.q, w.R, coeffs, w.r, w.z, w.scal, w.dinv, w.Rf, w.dinvf, w.bar, w.status,
                                  false, p->desc.solver == SFFT_SOLVE_PCG ? w.flags : nullptr, st);
    return e;
}

sfft_status sfft_normal(sfft_plan_t plan, const void *sci, const void *tmpl, const uint8_t *mask, double *N,
                        double *b) {
    sfft_status s = check_images(plan, sci, tmpl);
    if (s != SFFT_OK) return s;
    if (!N || !b) return set_err(plan, "null output pointer"), SFFT_ERR_INVALID_ARG;
    if (plan->profile) plan->timed_calls++;
    return queue_normal(plan, sci, tmpl, mask, N, b);
}

static sfft_status read_status(sfft_plan_t p, sfft_fit_info *info) {
    int st_h = 0, fl[3] = {0, 0, 0};
    double scal[3] = {0.0, 0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(&st_h, p->ws.status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scal, p->ws.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fl, p->ws.flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "status read-back");
    if (info) {
        memset(info, 0, sizeof *info);
        info->status = st_h;
        info->n = p->g.n;
        const bool fast = p->desc.solver == SFFT_SOLVE_PCG;
        info->iterations = fast && fl[0] ? fl[1] : 1;
        info->fallback = fast && !fl[0] ? 1 : 0;
        info->rel_residual = scal[1] > 0 ? sqrt(scal[0] / scal[1]) : 0.0;
        info->start_residual = fast && fl[0] && scal[1] > 0 ? sqrt(scal[2] / scal[1]) : 1.0;
        info->pcg_status = fast && !fl[0] ? (fl[2] ? fl[2] : (int)SFFT_ERR_NOT_SPD) : 0;
    }
    if (st_h != 0) {
        set_err(p, "device status: %s", sfft_status_string((sfft_status)st_h));
        cudaMemsetAsync(p->ws.status, 0, sizeof(int), p->stream);
    }
    return (sfft_status)st_h;
}

sfft_status sfft_fit(sfft_plan_t plan, const void *sci, const void *tmpl, const uint8_t *mask, const double *x0,
                     double *coeffs, sfft_fit_info *info) {
    (void)x0;
    sfft_status s = check_images(plan, sci, tmpl);
    if (s != SFFT_OK) return s;
    if (!coeffs) return set_err(plan, "null coeffs"), SFFT_ERR_INVALID_ARG;
    Workspace &w = plan->ws;
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(int), plan->stream);
    if (e != cudaSuccess) return cuda_fail(plan, e, "status reset");
    if (plan->profile) plan->timed_calls++;
    s = queue_normal(plan, sci, tmpl, mask, w.N, w.b);
    if (s != SFFT_OK) return s;
    {
        StageTimer t(plan, ST_SOLVE);
        const bool fast = plan->desc.solver == SFFT_SOLVE_PCG;
        e = cudaMemsetAsync(w.flags, 0, 3 * sizeof(int), plan->stream);
        if (e == cudaSuccess && fast && pcg_cluster_size(plan->g) > 0) {
            const int max_iter = plan->desc.max_iter > 0 ? plan->desc.max_iter : 50;
            const double tol = plan->desc.tol > 0.0 ? plan->desc.tol : 1e-12;
            e = launch_pcg_cluster(plan->g, w.N, w.b, x0, coeffs, w.r, w.p, w.q, w.z, w.dscale, w.Lg, w.scal, w.flags,
                                   max_iter, tol, false, plan->stream);
        }
        // FP64 Cholesky: the plain solver, or the fallback when PCG did not converge
        if (e == cudaSuccess) e = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), plan->stream);
        if (e == cudaSuccess)
            e = launch_cholesky_solve(plan->g, w.N, w.b, w.R, coeffs, w.r, w.z, w.scal, w.dinv, w.Rf, w.dinvf, w.bar,
                                      w.status, true, fast ? w.flags : nullptr, plan->stream);
    }
    if (e != cudaSuccess) return cuda_fail(plan, e, "solver launch");
    for (int pass = 0; pass < plan->g.refine; pass++) {
        StageTimer t(plan, ST_REFINE);
        e = queue_refine(plan, sci, tmpl, mask, coeffs);
        if (e != cudaSuccess) return cuda_fail(plan, e, "refinement launch");
    }
    if (e != cudaSuccess) return cuda_fail(plan, e, "solver launch");
    if (info) return read_status(plan, info);
    return SFFT_OK;
}

sfft_status sfft_subtract(sfft_plan_t plan, const void *sci, const void *tmpl, const double *coeffs, void *diff) {
    sfft_status s = check_images(plan, sci, tmpl);
    if (s != SFFT_OK) return s;
    if (!coeffs || !diff) return set_err(plan, "null coeffs or diff"), SFFT_ERR_INVALID_ARG;
    if (diff == sci || diff == tmpl) return set_err(plan, "diff may not alias the inputs"), SFFT_ERR_INVALID_ARG;
    cudaError_t e;
    {
        StageTimer t(plan, ST_SUBTRACT);
        // FP32 paths with subtract_fft tuned on: the row-segment FFT route where it has kernels
        // (DK <= 2, 3 <= L <= 15, DB <= 4); otherwise the direct kernel
        e = plan->desc.precision == SFFT_PREC_FP64 || !plan->g.subfft
                ? cudaErrorNotSupported
                : launch_subtract_fft(plan->g, plan->desc.dtype, sci, tmpl, coeffs, plan->ws.tw_fft, plan->ws.xpow,
                                      plan->ws.ypow, plan->ws.kspec, diff, plan->stream);
        if (e == cudaErrorNotSupported)
            e = launch_subtract(plan->g, plan->desc.dtype, plan->desc.precision, sci, tmpl, nullptr, false, coeffs,
                                plan->ws.xpow, plan->ws.ypow, plan->ws.cfold, diff, nullptr, nullptr, plan->stream);
    }
    if (e != cudaSuccess) return cuda_fail(plan, e, "subtract launch");
    return SFFT_OK;
}

sfft_status sfft_sync_status(sfft_plan_t plan) {
    if (!plan) return set_err(nullptr, "null plan"), SFFT_ERR_INVALID_ARG;
    return read_status(plan, nullptr);
}


}  // extern "C"
