// Cross-convolution by row-segment FFTs (Sec. "Pipeline steps", steps 5 and 7): the same
// cyclic convolution as the direct kernel of sfft_xconv.cu,
//   out(y, x) = sum_{a,b} P[a][b] X((y - a + r) mod Ny, (x - b + r) mod Nx),  K = 2r + 1,
// computed per 256-column segment.  Segment s owns the output columns [x0, x0 + U),
// U = 256 - 2r, and reads the cyclic input window Z_y(j) = X(y, x0 - r + j), j < 256.  For
// i < U the 256-point cyclic convolution of Z with stamp row p_a(m) = P[a][m] at n = i + 2r
// only touches j = n - m in [i, i + 2r], inside the window, so
//   out(y, x0 + i) = IDFT_256( sum_a Phat_a(k) Zhat_{y - a + r}(k) )(i + 2r).
// One CTA takes one segment of one image and a run of 32-row chunks:
//   1. the stamp rows' DFTs Phat_a (two real rows per complex FFT), scaled by 1/256;
//   2. per chunk, the DFTs of its 32 + 2r input rows (two rows per complex FFT) into shared
//      memory, 128 slots per row (slot 0 packs the real bins 0 and 128);
//   3. the K-tap correlation over rows per frequency slot, FP32 in registers (two threads
//      per slot, 16 output rows each, the stamp rows in two passes);
//   4. the inverse DFTs of the output rows (two rows per complex FFT), written to the frame.
// About 70 instructions per output pixel against ~800 for the direct K^2 = 625-tap sum.
// FP32 with split (hi + lo) twiddles, so FFT rounding stays near 1e-7 of the row's scale.
#include <math.h>
#include <stdio.h>

#include "sfft_rowfft.cuh"

namespace sfft {

int device_sm_count();

namespace {

constexpr int kXThreads = 256;  // 16 half-warps; the first kXFft of them run the 256-point FFTs
constexpr int kXFft = 8;        // FFTs in flight (exchange buffers): two CTAs fit an SM
constexpr int kXChunk = 32;     // output rows per chunk

template <int R>
struct XF {
    static constexpr int K = 2 * R + 1, U = kP - 2 * R, NIN = kXChunk + 2 * R;
    static constexpr int NA = (K + 1) / 2;  // stamp rows in the first MAC pass
};

// shared memory: split twiddles, 16 exchange buffers, the stamp table [K][128] and the
// chunk's spectra [NIN][128] (input rows, then the output rows in the first 32 slots)
template <int R>
struct XSmem {
    static constexpr size_t tw = 0;
    static constexpr size_t ex = tw + 2 * kP * sizeof(cpx<float>);
    static constexpr size_t ptab = ex + kXFft * (size_t)kXEx * sizeof(cpx<float>);
    static constexpr size_t spec = ptab + (size_t)XF<R>::K * 128 * sizeof(float2);
    static constexpr size_t bytes = spec + (size_t)XF<R>::NIN * 128 * sizeof(float2);
};

// One MAC pass over stamp rows a in [A0, A1): acc[jj] += Phat_a(slot) Zhat_{j0 + jj + 2r - a}(slot)
// for the thread's 16 output rows.  Complex products as two packed FMAs:
// z p = (z.re, z.re)(p.re, p.im) + (z.im, z.im)(-p.im, p.re); slot 0 holds the real bins 0 and
// 128 side by side, whose products are elementwise: (z.x, z.y)(p.x, p.y) + 0.
template <int R, int A0, int A1>
__device__ __forceinline__ void mac_pass(const float2 *spec, const float2 *ptab, int slot, int j0, bool packed,
                                         float2 (&acc)[16]) {
    constexpr int NA = A1 - A0;
    float2 p[NA], pn[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) {
        const float2 q = ptab[(A0 + a) * 128 + slot];
        p[a] = q;
        pn[a] = packed ? make_float2(0.f, 0.f) : make_float2(-q.y, q.x);
    }
#pragma unroll
    for (int d = -(A1 - 1); d <= 15 - A0; d++) {
        const float2 z = spec[(j0 + 2 * R + d) * 128 + slot];
        const float2 za = make_float2(z.x, packed ? z.y : z.x), zb = make_float2(z.y, z.y);
#pragma unroll
        for (int a = A0; a < A1; a++) {
            const int jj = d + a;
            if (jj >= 0 && jj < 16) {
                acc[jj] = __ffma2_rn(za, p[a - A0], acc[jj]);
                acc[jj] = __ffma2_rn(zb, pn[a - A0], acc[jj]);
            }
        }
    }
}

struct XJobF {
    const void *src;
    const float *psf;
    void *dst;
};

template <class In, int R>
__global__ void __launch_bounds__(kXThreads, XSmem<R>::bytes <= 113 * 1024 ? 2 : 1) k_xconv_fft(XJobF j0, XJobF j1, int ny, int nx, int pitch) {
    using F = XF<R>;
    using SM = XSmem<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float> *tw = reinterpret_cast<cpx<float> *>(smem_raw + SM::tw);
    float2 *ptab = reinterpret_cast<float2 *>(smem_raw + SM::ptab);
    float2 *spec = reinterpret_cast<float2 *>(smem_raw + SM::spec);
    const XJobF jb = blockIdx.z ? j1 : j0;
    const In *src = reinterpret_cast<const In *>(jb.src);
    In *dst = reinterpret_cast<In *>(jb.dst);
    const int x0 = blockIdx.x * F::U, t = threadIdx.x, hw = t >> 4, lt = t & 15;
    const unsigned msk = (hw & 1) ? 0xffff0000u : 0x0000ffffu;
    const bool fft_lane = hw < kXFft;  // half-warps that run FFTs
    cpx<float> *e = reinterpret_cast<cpx<float> *>(smem_raw + SM::ex) + (hw % kXFft) * kXEx;
    // split twiddles exp(-2 pi i m / 256) = wh + wl of the FP32 FFT's per-(k1, lane) table
    // (tw4 entry i holds m = (i / 16 + 1) (i mod 16)), in the tw / twl bytes
    float4 *tw4 = reinterpret_cast<float4 *>(tw);
    for (int i = t; i < kTw4; i += kXThreads) {
        const int m = ((i >> 4) + 1) * (i & 15);
        double sn, cs;
        sincospi(-2.0 * m / kP, &sn, &cs);
        const float ch = (float)cs, sh = (float)sn;
        tw4[i] = make_float4(ch, sh, (float)(cs - (double)ch), (float)(sn - (double)sh));
    }
    __syncthreads();
    // 1. the stamp rows' spectra, with the inverse transform's 1/256
    for (int pa = hw; fft_lane && 2 * pa < F::K; pa += kXFft) {
        const int a1 = 2 * pa, a2 = 2 * pa + 1;
        cpx<float> v[16];
#pragma unroll
        for (int jj = 0; jj < 16; jj++) {
            const int m = lt + 16 * jj;
            v[jj].re = m < F::K ? jb.psf[a1 * F::K + m] : 0.f;
            v[jj].im = (m < F::K && a2 < F::K) ? jb.psf[a2 * F::K + m] : 0.f;
        }
        fft256f(v, lt, e, tw4, msk);
        unpack_pair(v, lt, e, ptab + a1 * 128, a2 < F::K ? ptab + a2 * 128 : nullptr, 1.f / kP, msk);
    }
    __syncthreads();
    const int slot = t >> 1, jh = 16 * (t & 1);
    const bool packed = slot == 0;
    const int nchunks = (ny + kXChunk - 1) / kXChunk;
    for (int c = blockIdx.y; c < nchunks; c += gridDim.y) {
        const int y0 = c * kXChunk;
        // 2. the chunk's input rows y0 - r .. y0 + 31 + r, two to a complex FFT
        // (the next pair's rows are loaded while the current one is transformed)
        constexpr int NPAIR = (F::NIN + 1) / 2;
        auto load_rows = [&](int pr, cpx<float>(&v)[16]) {
            const int r1 = 2 * pr, r2 = 2 * pr + 1;
            int yy1 = (y0 - R + r1) % ny, yy2 = (y0 - R + r2) % ny;
            yy1 += yy1 < 0 ? ny : 0;
            yy2 += yy2 < 0 ? ny : 0;
            load_pair<In>(src + (size_t)yy1 * pitch, r2 < F::NIN ? src + (size_t)yy2 * pitch : nullptr, x0 - R, nx, lt,
                          v);
        };
        cpx<float> vn[16];
        if (fft_lane && hw < NPAIR) load_rows(hw, vn);
        for (int pr = hw; fft_lane && pr < NPAIR; pr += kXFft) {
            cpx<float> v[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) v[jj] = vn[jj];
            if (pr + kXFft < NPAIR) load_rows(pr + kXFft, vn);
            fft256f(v, lt, e, tw4, msk);
            const int r1 = 2 * pr, r2 = r1 + 1;
            unpack_pair(v, lt, e, spec + r1 * 128, r2 < F::NIN ? spec + r2 * 128 : nullptr, 1.f, msk);
        }
        __syncthreads();
        // 3. the K-tap correlation over rows for this thread's slot and 16 output rows
        float2 acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; jj++) acc[jj] = make_float2(0.f, 0.f);
        mac_pass<R, 0, F::NA>(spec, ptab, slot, jh, packed, acc);
        if constexpr (F::NA < F::K) mac_pass<R, F::NA, F::K>(spec, ptab, slot, jh, packed, acc);
        __syncthreads();  // every input slot read
#pragma unroll
        for (int jj = 0; jj < 16; jj++) spec[(jh + jj) * 128 + slot] = acc[jj];
        __syncthreads();
        // 4. output rows 2 op, 2 op + 1 for the FFT half-warps' pairs op: y = conj(FFT(conj(Y1 + i Y2)))
        for (int op = hw; fft_lane && op < kXChunk / 2; op += kXFft) {
            const int o1 = 2 * op, o2 = o1 + 1;
            const float2 *Y1 = spec + o1 * 128, *Y2 = spec + o2 * 128;
            cpx<float> v[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int n = lt + 16 * jj;
                const float2 a = half_bin(Y1, n), b = half_bin(Y2, n);
                v[jj] = {a.x - b.y, -(a.y + b.x)};
            }
            fft256f(v, lt, e, tw4, msk);
#pragma unroll
            for (int k2 = 0; k2 < 16; k2++) {
                const int i = lt + 16 * k2 - 2 * R;
                if (i < 0 || i >= F::U || x0 + i >= nx) continue;
                if (y0 + o1 < ny) dst[(size_t)(y0 + o1) * pitch + x0 + i] = (In)v[k2].re;
                if (y0 + o2 < ny) dst[(size_t)(y0 + o2) * pitch + x0 + i] = (In)(-v[k2].im);
            }
        }
        __syncthreads();  // the next chunk overwrites the spectra
    }
}

template <class In, int R>
cudaError_t run_fft_r(const XJobF &a, const XJobF &b, int njobs, int ny, int nx, int pitch, cudaStream_t st) {
    using SM = XSmem<R>;
    auto kern = k_xconv_fft<In, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e != cudaSuccess) return e;
    // segments x chunk groups x images: one wave of two CTAs per SM (one for the largest
    // stamps, whose tables do not fit twice), each CTA a run of chunks
    const int nseg = (nx + XF<R>::U - 1) / XF<R>::U, nchunks = (ny + kXChunk - 1) / kXChunk;
    int groups = device_sm_count() * (SM::bytes <= 113 * 1024 ? 2 : 1) / (nseg * njobs);  // CTAs per SM as in the launch bounds
    groups = groups < 1 ? 1 : (groups > nchunks ? nchunks : groups);
    dim3 grid(nseg, groups, njobs);
    note_launch();
    kern<<<grid, kXThreads, SM::bytes, st>>>(a, b, ny, nx, pitch);
    return cudaGetLastError();
}

template <class In>
cudaError_t run_fft_in(int r, const XJobF &a, const XJobF &b, int njobs, int ny, int nx, int pitch, cudaStream_t st) {
    switch (r) {
        case 4: return run_fft_r<In, 4>(a, b, njobs, ny, nx, pitch, st);
        case 5: return run_fft_r<In, 5>(a, b, njobs, ny, nx, pitch, st);
        case 6: return run_fft_r<In, 6>(a, b, njobs, ny, nx, pitch, st);
        case 7: return run_fft_r<In, 7>(a, b, njobs, ny, nx, pitch, st);
        case 8: return run_fft_r<In, 8>(a, b, njobs, ny, nx, pitch, st);
        case 9: return run_fft_r<In, 9>(a, b, njobs, ny, nx, pitch, st);
        case 10: return run_fft_r<In, 10>(a, b, njobs, ny, nx, pitch, st);
        case 11: return run_fft_r<In, 11>(a, b, njobs, ny, nx, pitch, st);
        case 12: return run_fft_r<In, 12>(a, b, njobs, ny, nx, pitch, st);
        case 13: return run_fft_r<In, 13>(a, b, njobs, ny, nx, pitch, st);
        case 14: return run_fft_r<In, 14>(a, b, njobs, ny, nx, pitch, st);
        case 15: return run_fft_r<In, 15>(a, b, njobs, ny, nx, pitch, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// the FFT route of the cross-convolution for stamp radii 4 .. 15 (K = 9 .. 31)
cudaError_t launch_xconv_fft(int r, int dtype, const void *src0, const float *psf0, void *dst0, const void *src1,
                             const float *psf1, void *dst1, int njobs, int ny, int nx, int pitch, cudaStream_t st) {
    const XJobF a{src0, psf0, dst0}, b{src1, psf1, dst1};
    return dtype == SFFT_F64 ? run_fft_in<double>(r, a, b, njobs, ny, nx, pitch, st)
                             : run_fft_in<float>(r, a, b, njobs, ny, nx, pitch, st);
}

}  // namespace sfft
