// Warm-start network: maps the PSF stamps of a science/template pair (9 grid cells x
// {science, template}, 32 x 32 each) to the delta-basis kernel coefficients of the fit,
// which the PCG solve takes as its starting point.  Layers: 4 x [3x3 convolution, stride 2,
// zero padding 1, 32 channels, ReLU] (32 -> 16 -> 8 -> 4 -> 2 px), flatten (channel, row,
// column), linear 128 -> n_out.  Training minimises the mean squared error against fitted
// coefficients with Adam (Kingma & Ba 2015, Algorithm 1; beta1 0.9, beta2 0.999, eps 1e-8).
//
// The network is small (126k parameters, ~2.2 M multiply-adds per sample), so every layer
// is a direct SIMT kernel: one thread per output value for the forward and input-gradient
// passes, one CTA per (output, input) channel pair for the weight gradients (a tree
// reduction over batch and pixels, deterministic).  All arithmetic is FP32; the loss is
// summed in FP64.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sfft_internal.cuh"

namespace sfft {
void set_global_error(const char *msg);
namespace {

constexpr int kIn = 18, kHW = 32, kCh = 32, kConv = 4, kFlat = 128;
constexpr float kB1 = 0.9f, kB2 = 0.999f, kEps = 1e-8f;

struct Layout {
    size_t w[kConv], b[kConv], wl, bl, total;
    int cin[kConv], hin[kConv];
};

Layout make_layout(int n_out) {
    Layout L{};
    size_t k = 0;
    for (int l = 0; l < kConv; l++) {
        L.cin[l] = l == 0 ? kIn : kCh;
        L.hin[l] = kHW >> l;
        L.w[l] = k;
        k += (size_t)kCh * L.cin[l] * 9;
        L.b[l] = k;
        k += kCh;
    }
    L.wl = k;
    k += (size_t)n_out * kFlat;
    L.bl = k;
    k += n_out;
    L.total = k;
    return L;
}

// a[n][o][i][j] = max(0, b[o] + sum_{c,u,v} W[o][c][u][v] x[n][c][2i+u-1][2j+v-1])
__global__ void k_conv_fwd(const float *__restrict__ x, int cin, int hin, const float *__restrict__ W,
                           const float *__restrict__ b, float *__restrict__ a, int B) {
    const int ho = hin >> 1;
    const long total = (long)B * kCh * ho * ho;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int j = (int)(t % ho), i = (int)((t / ho) % ho), o = (int)((t / ((long)ho * ho)) % kCh);
        const long n = t / ((long)ho * ho * kCh);
        float z = b[o];
        for (int c = 0; c < cin; c++) {
            const float *xc = x + ((n * cin + c) * hin) * hin;
            const float *wc = W + ((size_t)o * cin + c) * 9;
#pragma unroll
            for (int u = 0; u < 3; u++) {
                const int yy = 2 * i + u - 1;
                if (yy < 0 || yy >= hin) continue;
#pragma unroll
                for (int v = 0; v < 3; v++) {
                    const int xx = 2 * j + v - 1;
                    if (xx < 0 || xx >= hin) continue;
                    z = fmaf(wc[u * 3 + v], xc[yy * hin + xx], z);
                }
            }
        }
        a[t] = fmaxf(z, 0.f);
    }
}

// out[n][k] = bl[k] + sum_j Wl[k][j] flat[n][j]
__global__ void k_linear_fwd(const float *__restrict__ flat, const float *__restrict__ Wl,
                             const float *__restrict__ bl, float *__restrict__ out, int B, int n_out) {
    const long total = (long)B * n_out;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int k = (int)(t % n_out);
        const long n = t / n_out;
        const float *w = Wl + (size_t)k * kFlat, *f = flat + n * kFlat;
        float s = bl[k];
#pragma unroll 8
        for (int j = 0; j < kFlat; j++) s = fmaf(w[j], f[j], s);
        out[t] = s;
    }
}

// loss = mean (out - t)^2 (FP64 sum), gout = 2 (out - t) / count; one CTA
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ tgt, float *__restrict__ gout,
                      long count, float *__restrict__ loss, float *__restrict__ loss_sum) {
    __shared__ double red[32];
    double acc = 0.0;
    const float sc = (float)(2.0 / (double)count);
    for (long e = threadIdx.x; e < count; e += blockDim.x) {
        const float d = out[e] - tgt[e];
        gout[e] = sc * d;
        acc += (double)d * (double)d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        const float l = (float)(s / (double)count);
        if (loss) loss[0] = l;
        if (loss_sum) loss_sum[0] += l;
    }
}

// gWl[k][j] = sum_n gout[n][k] flat[n][j]; gbl[k] = sum_n gout[n][k] (column j == kFlat)
__global__ void k_linear_bwd_w(const float *__restrict__ gout, const float *__restrict__ flat,
                               float *__restrict__ gWl, float *__restrict__ gbl, int B, int n_out) {
    const long total = (long)n_out * (kFlat + 1);
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int j = (int)(t % (kFlat + 1)), k = (int)(t / (kFlat + 1));
        float s = 0.f;
        for (int n = 0; n < B; n++) s = fmaf(gout[(size_t)n * n_out + k], j < kFlat ? flat[(size_t)n * kFlat + j] : 1.f, s);
        if (j < kFlat)
            gWl[(size_t)k * kFlat + j] = s;
        else
            gbl[k] = s;
    }
}

// gflat[n][j] = sum_k Wl[k][j] gout[n][k]
__global__ void k_linear_bwd_x(const float *__restrict__ gout, const float *__restrict__ Wl,
                               float *__restrict__ gflat, int B, int n_out) {
    const long total = (long)B * kFlat;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int j = (int)(t % kFlat);
        const long n = t / kFlat;
        float s = 0.f;
        for (int k = 0; k < n_out; k++) s = fmaf(Wl[(size_t)k * kFlat + j], gout[n * n_out + k], s);
        gflat[t] = s;
    }
}

// weight and bias gradients of one convolution: one CTA per (o, c); gz = ga where a > 0
__global__ void k_conv_bwd_w(const float *__restrict__ x, int cin, int hin, const float *__restrict__ a,
                             const float *__restrict__ ga, float *__restrict__ gW, float *__restrict__ gb, int B) {
    const int c = blockIdx.x, o = blockIdx.y, ho = hin >> 1;
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; k++) acc[k] = 0.f;
    const long total = (long)B * ho * ho;
    for (long t = threadIdx.x; t < total; t += blockDim.x) {
        const int j = (int)(t % ho), i = (int)((t / ho) % ho);
        const long n = t / ((long)ho * ho);
        const long ia = ((n * kCh + o) * ho + i) * ho + j;
        const float gz = a[ia] > 0.f ? ga[ia] : 0.f;
        const float *xc = x + ((n * cin + c) * hin) * hin;
#pragma unroll
        for (int u = 0; u < 3; u++) {
            const int yy = 2 * i + u - 1;
#pragma unroll
            for (int v = 0; v < 3; v++) {
                const int xx = 2 * j + v - 1;
                if (yy >= 0 && yy < hin && xx >= 0 && xx < hin) acc[u * 3 + v] = fmaf(gz, xc[yy * hin + xx], acc[u * 3 + v]);
            }
        }
        acc[9] += gz;
    }
    __shared__ float red[10][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; k++) {
        float s = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) red[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        float s = 0.f;
        for (int w = 0; w < nw; w++) s += red[threadIdx.x][w];
        if (threadIdx.x < 9)
            gW[((size_t)o * cin + c) * 9 + threadIdx.x] = s;
        else if (c == 0)
            gb[o] = s;
    }
}

// input gradient of one convolution: gx[n][c][y][x] = sum_{o,u,v} W[o][c][u][v] gz[n][o][i][j]
// over the (i, j) with 2i + u - 1 = y, 2j + v - 1 = x
__global__ void k_conv_bwd_x(const float *__restrict__ W, int cin, int hin, const float *__restrict__ a,
                             const float *__restrict__ ga, float *__restrict__ gx, int B) {
    const int ho = hin >> 1;
    const long total = (long)B * cin * hin * hin;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int xx = (int)(t % hin), yy = (int)((t / hin) % hin), c = (int)((t / ((long)hin * hin)) % cin);
        const long n = t / ((long)hin * hin * cin);
        float s = 0.f;
        for (int u = 0; u < 3; u++) {
            const int iy = yy + 1 - u;
            if (iy < 0 || (iy & 1) || (iy >> 1) >= ho) continue;
            const int i = iy >> 1;
            for (int v = 0; v < 3; v++) {
                const int ix = xx + 1 - v;
                if (ix < 0 || (ix & 1) || (ix >> 1) >= ho) continue;
                const int j = ix >> 1;
                for (int o = 0; o < kCh; o++) {
                    const long ia = ((n * kCh + o) * ho + i) * ho + j;
                    const float gz = a[ia] > 0.f ? ga[ia] : 0.f;
                    s = fmaf(W[((size_t)o * cin + c) * 9 + u * 3 + v], gz, s);
                }
            }
        }
        gx[t] = s;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long count, float lr, float bc1, float bc2) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = kB1 * m[t] + (1.f - kB1) * gt;
        const float vt = kB2 * v[t] + (1.f - kB2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        p[t] -= lr * (mt / bc1) / (sqrtf(vt / bc2) + kEps);
    }
}

__global__ void k_gather(const float *__restrict__ src, const int *__restrict__ idx, long per,
                         float *__restrict__ dst, int B) {
    const long total = (long)B * per;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long b = t / per, e = t - b * per;
        dst[t] = src[(long)idx[b] * per + e];
    }
}

__global__ void k_warm(const float *__restrict__ out, int B, int n_out, int n_stride, double *__restrict__ x0) {
    const long total = (long)B * n_stride;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long b = t / n_stride;
        const int j = (int)(t - b * n_stride);
        x0[t] = j < n_out ? (double)out[b * n_out + j] : 0.0;
    }
}

unsigned blocks_for(long n, int threads = 256) {
    long b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 65535L * 4 ? 65535L * 4 : b));
}

// SplitMix64 (Steele, Lea & Flood 2014): the host PRNG that shuffles minibatches
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace sfft

using namespace sfft;

struct sfft_cnn_s {
    int n_out = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    Layout lay{};
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *act[kConv] = {}, *gact[kConv] = {};
    float *out = nullptr, *gout = nullptr, *xb = nullptr, *tb = nullptr, *loss = nullptr;
    int *idx = nullptr;
    long step = 0;
    void *block = nullptr;
    char err[256] = {0};
};

namespace {

sfft_status cnn_err(sfft_cnn_t c, sfft_status s, const char *msg) {
    if (c) snprintf(c->err, sizeof c->err, "%s", msg);
    set_global_error(msg);
    return s;
}

sfft_status cnn_cuda(sfft_cnn_t c, cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return cnn_err(c, SFFT_ERR_CUDA, buf);
}

// forward pass of `B` samples at x into c->act / c->out
cudaError_t forward(sfft_cnn_t c, const float *x, int B) {
    const Layout &L = c->lay;
    const float *in = x;
    for (int l = 0; l < kConv; l++) {
        const int ho = L.hin[l] >> 1;
        note_launch();
        k_conv_fwd<<<blocks_for((long)B * kCh * ho * ho), 256, 0, c->stream>>>(
            in, L.cin[l], L.hin[l], c->params + L.w[l], c->params + L.b[l], c->act[l], B);
        in = c->act[l];
    }
    note_launch();
    k_linear_fwd<<<blocks_for((long)B * c->n_out), 256, 0, c->stream>>>(c->act[kConv - 1], c->params + L.wl,
                                                                        c->params + L.bl, c->out, B, c->n_out);
    return cudaGetLastError();
}

// loss and gradients (into c->grad, and the input gradient into gin when non-null)
cudaError_t backward(sfft_cnn_t c, const float *x, const float *tgt, int B, float *gin, float *loss_sum) {
    const Layout &L = c->lay;
    note_launch();
    k_mse<<<1, 1024, 0, c->stream>>>(c->out, tgt, c->gout, (long)B * c->n_out, c->loss, loss_sum);
    note_launch();
    k_linear_bwd_w<<<blocks_for((long)c->n_out * (kFlat + 1)), 256, 0, c->stream>>>(
        c->gout, c->act[kConv - 1], c->grad + L.wl, c->grad + L.bl, B, c->n_out);
    note_launch();
    k_linear_bwd_x<<<blocks_for((long)B * kFlat), 256, 0, c->stream>>>(c->gout, c->params + L.wl,
                                                                       c->gact[kConv - 1], B, c->n_out);
    for (int l = kConv - 1; l >= 0; l--) {
        const float *xin = l ? c->act[l - 1] : x;
        note_launch();
        k_conv_bwd_w<<<dim3(L.cin[l], kCh), 256, 0, c->stream>>>(xin, L.cin[l], L.hin[l], c->act[l], c->gact[l],
                                                                 c->grad + L.w[l], c->grad + L.b[l], B);
        float *gx = l ? c->gact[l - 1] : gin;
        if (gx) {
            note_launch();
            k_conv_bwd_x<<<blocks_for((long)B * L.cin[l] * L.hin[l] * L.hin[l]), 256, 0, c->stream>>>(
                c->params + L.w[l], L.cin[l], L.hin[l], c->act[l], c->gact[l], gx, B);
        }
    }
    return cudaGetLastError();
}

cudaError_t adam(sfft_cnn_t c, float lr) {
    c->step++;
    const double bc1 = 1.0 - std::pow((double)kB1, (double)c->step);
    const double bc2 = 1.0 - std::pow((double)kB2, (double)c->step);
    note_launch();
    k_adam<<<blocks_for((long)c->lay.total), 256, 0, c->stream>>>(c->params, c->grad, c->m, c->v, (long)c->lay.total,
                                                                  lr, (float)bc1, (float)bc2);
    return cudaGetLastError();
}

sfft_status check_batch(sfft_cnn_t c, int B) {
    if (!c) return cnn_err(nullptr, SFFT_ERR_INVALID_ARG, "null network");
    if (B < 1 || B > c->max_batch) {
        char buf[128];
        snprintf(buf, sizeof buf, "batch %d outside [1, %d]", B, c->max_batch);
        return cnn_err(c, SFFT_ERR_INVALID_ARG, buf);
    }
    return SFFT_OK;
}

}  // namespace

extern "C" {

sfft_status sfft_cnn_create(sfft_cnn_t *out, int32_t n_out, int32_t max_batch, sfft_stream_t stream) {
    if (!out) return cnn_err(nullptr, SFFT_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (n_out < 1 || max_batch < 1) return cnn_err(nullptr, SFFT_ERR_INVALID_ARG, "n_out and max_batch must be >= 1");
    sfft_cnn_t c = new sfft_cnn_s;
    c->n_out = n_out;
    c->max_batch = max_batch;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->lay = make_layout(n_out);
    const size_t P = c->lay.total, B = (size_t)max_batch;
    size_t act = 0;
    for (int l = 0; l < kConv; l++) act += B * kCh * (size_t)(kHW >> (l + 1)) * (kHW >> (l + 1));
    const size_t floats = 4 * P + 2 * act + 2 * B * n_out + B * kIn * kHW * kHW + B * n_out + 2;
    const size_t bytes = floats * sizeof(float) + B * sizeof(int) + 256;
    cudaError_t e = cudaMalloc(&c->block, bytes);
    if (e != cudaSuccess) {
        delete c;
        return cnn_err(nullptr, SFFT_ERR_OOM, "network workspace allocation failed");
    }
    float *f = static_cast<float *>(c->block);
    c->params = f, f += P;
    c->grad = f, f += P;
    c->m = f, f += P;
    c->v = f, f += P;
    for (int l = 0; l < kConv; l++) {
        const size_t s = B * kCh * (size_t)(kHW >> (l + 1)) * (kHW >> (l + 1));
        c->act[l] = f, f += s;
        c->gact[l] = f, f += s;
    }
    c->out = f, f += B * n_out;
    c->gout = f, f += B * n_out;
    c->xb = f, f += B * kIn * kHW * kHW;
    c->tb = f, f += B * n_out;
    c->loss = f, f += 2;
    c->idx = reinterpret_cast<int *>(f);
    e = cudaMemsetAsync(c->block, 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(c->block);
        delete c;
        return cnn_cuda(nullptr, e, "network workspace initialisation");
    }
    *out = c;
    return SFFT_OK;
}

void sfft_cnn_destroy(sfft_cnn_t c) {
    if (!c) return;
    if (c->block) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->block);
    }
    delete c;
}

sfft_status sfft_cnn_param_count(sfft_cnn_t c, int64_t *count) {
    if (!c || !count) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    *count = (int64_t)c->lay.total;
    return SFFT_OK;
}

sfft_status sfft_cnn_set_params(sfft_cnn_t c, const float *params) {
    if (!c || !params) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    const size_t P = c->lay.total;
    cudaError_t e = cudaMemcpyAsync(c->params, params, P * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, 2 * P * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda(c, e, "set_params");
    c->step = 0;
    return SFFT_OK;
}

sfft_status sfft_cnn_get_params(sfft_cnn_t c, float *params) {
    if (!c || !params) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpyAsync(params, c->params, c->lay.total * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda(c, e, "get_params");
    return SFFT_OK;
}

static const char kCnnTag[8] = {'S', 'F', 'F', 'T', 'C', 'N', 'N', '1'};

sfft_status sfft_cnn_save(sfft_cnn_t c, const char *path) {
    if (!c || !path) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    const int64_t P = (int64_t)c->lay.total;
    std::vector<float> h((size_t)P);
    sfft_status s = sfft_cnn_get_params(c, h.data());
    if (s != SFFT_OK) return s;
    FILE *f = fopen(path, "wb");
    if (!f) return cnn_err(c, SFFT_ERR_INVALID_ARG, "save: cannot open the file for writing");
    const int32_t hdr[2] = {c->n_out, 0};
    bool ok = fwrite(kCnnTag, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 && fwrite(&P, sizeof P, 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), (size_t)P, f) == (size_t)P;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return cnn_err(c, SFFT_ERR_INVALID_ARG, "save: write failed");
    return SFFT_OK;
}

sfft_status sfft_cnn_load(sfft_cnn_t c, const char *path) {
    if (!c || !path) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    FILE *f = fopen(path, "rb");
    if (!f) return cnn_err(c, SFFT_ERR_INVALID_ARG, "load: cannot open the file");
    char tag[8];
    int32_t hdr[2];
    int64_t P = 0;
    const int64_t want = (int64_t)c->lay.total;
    bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, kCnnTag, 8) == 0 && fread(hdr, sizeof hdr, 1, f) == 1 &&
              fread(&P, sizeof P, 1, f) == 1;
    if (!ok) {
        fclose(f);
        return cnn_err(c, SFFT_ERR_INVALID_ARG, "load: not a network file");
    }
    if (hdr[0] != c->n_out || P != want) {
        fclose(f);
        return cnn_err(c, SFFT_ERR_INVALID_ARG, "load: the file's output width or parameter count differs");
    }
    std::vector<float> h((size_t)P);
    ok = fread(h.data(), sizeof(float), (size_t)P, f) == (size_t)P;
    char extra;
    ok = ok && fread(&extra, 1, 1, f) == 0;  // nothing after the parameters
    fclose(f);
    if (!ok) return cnn_err(c, SFFT_ERR_INVALID_ARG, "load: short or oversized file");
    return sfft_cnn_set_params(c, h.data());
}

sfft_status sfft_cnn_forward(sfft_cnn_t c, const float *stamps, int32_t batch, float *out) {
    sfft_status s = check_batch(c, batch);
    if (s != SFFT_OK) return s;
    if (!stamps || !out) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    cudaError_t e = forward(c, stamps, batch);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->out, (size_t)batch * c->n_out * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cnn_cuda(c, e, "forward");
    return SFFT_OK;
}

sfft_status sfft_cnn_gradients(sfft_cnn_t c, const float *stamps, const float *targets, int32_t batch, float *grad,
                               float *grad_in, float *loss) {
    sfft_status s = check_batch(c, batch);
    if (s != SFFT_OK) return s;
    if (!stamps || !targets || !grad) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument");
    cudaError_t e = forward(c, stamps, batch);
    if (e == cudaSuccess) e = backward(c, stamps, targets, batch, grad_in, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad, c->grad, c->lay.total * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, c->loss, sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cnn_cuda(c, e, "gradients");
    return SFFT_OK;
}

sfft_status sfft_cnn_train_step(sfft_cnn_t c, const float *stamps, const float *targets, int32_t batch, float lr,
                                float *loss) {
    sfft_status s = check_batch(c, batch);
    if (s != SFFT_OK) return s;
    if (!stamps || !targets || !(lr > 0.f)) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument or lr <= 0");
    cudaError_t e = forward(c, stamps, batch);
    if (e == cudaSuccess) e = backward(c, stamps, targets, batch, nullptr, nullptr);
    if (e == cudaSuccess) e = adam(c, lr);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, c->loss, sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cnn_cuda(c, e, "train_step");
    return SFFT_OK;
}

sfft_status sfft_cnn_train(sfft_cnn_t c, const float *stamps, const float *targets, int32_t n, int32_t batch,
                           int32_t epochs, float lr, uint64_t seed, float *epoch_loss) {
    sfft_status s = check_batch(c, batch);
    if (s != SFFT_OK) return s;
    if (!stamps || !targets || n < batch || epochs < 1 || !(lr > 0.f))
        return cnn_err(c, SFFT_ERR_INVALID_ARG, "null data, n < batch, epochs < 1 or lr <= 0");
    std::vector<int> order(n);
    uint64_t st = seed;
    const long per_x = (long)kIn * kHW * kHW;
    const int steps = n / batch;  // the ragged remainder of each shuffled epoch is skipped
    for (int ep = 0; ep < epochs; ep++) {
        for (int i = 0; i < n; i++) order[i] = i;
        for (int i = n - 1; i > 0; i--) {  // Fisher-Yates
            const int j = (int)(splitmix64(st) % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        cudaError_t e = cudaMemsetAsync(c->loss + 1, 0, sizeof(float), c->stream);
        for (int k = 0; k < steps && e == cudaSuccess; k++) {
            // a copy from pageable memory is staged before the call returns; stream order
            // keeps the next copy behind this batch's gathers
            e = cudaMemcpyAsync(c->idx, order.data() + (size_t)k * batch, (size_t)batch * sizeof(int),
                                cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) {
                note_launch();
                k_gather<<<blocks_for((long)batch * per_x), 256, 0, c->stream>>>(stamps, c->idx, per_x, c->xb, batch);
                note_launch();
                k_gather<<<blocks_for((long)batch * c->n_out), 256, 0, c->stream>>>(targets, c->idx, c->n_out, c->tb,
                                                                                    batch);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = forward(c, c->xb, batch);
            if (e == cudaSuccess) e = backward(c, c->xb, c->tb, batch, nullptr, c->loss + 1);
            if (e == cudaSuccess) e = adam(c, lr);
        }
        float sum = 0.f;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&sum, c->loss + 1, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cnn_cuda(c, e, "train");
        if (epoch_loss) epoch_loss[ep] = sum / (float)steps;
    }
    return SFFT_OK;
}

sfft_status sfft_cnn_warm_start(sfft_cnn_t c, const float *stamps, int32_t batch, int32_t n_stride, double *x0) {
    sfft_status s = check_batch(c, batch);
    if (s != SFFT_OK) return s;
    if (!stamps || !x0 || n_stride < c->n_out) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null argument or n_stride < n_out");
    cudaError_t e = forward(c, stamps, batch);
    if (e == cudaSuccess) {
        note_launch();
        k_warm<<<blocks_for((long)batch * n_stride), 256, 0, c->stream>>>(c->out, batch, c->n_out, n_stride, x0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cnn_cuda(c, e, "warm_start");
    return SFFT_OK;
}

sfft_status sfft_cnn_set_stream(sfft_cnn_t c, sfft_stream_t stream) {
    if (!c) return cnn_err(c, SFFT_ERR_INVALID_ARG, "null network");
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    return SFFT_OK;
}

const char *sfft_cnn_last_error(sfft_cnn_t c) { return c ? c->err : sfft_last_error(nullptr); }

}  // extern "C"

namespace sfft {
int cnn_n_out(sfft_cnn_t c) { return c ? c->n_out : -1; }
int cnn_max_batch(sfft_cnn_t c) { return c ? c->max_batch : 0; }
cudaStream_t cnn_stream(sfft_cnn_t c) { return c ? c->stream : nullptr; }
}  // namespace sfft
