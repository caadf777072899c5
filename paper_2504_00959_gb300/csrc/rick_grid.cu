// rick_grid.cu -- convolutional gridding, Eq. 3 of the paper (sub-step 2 of
// step 2 in Sec. 2.1), and the taper used for grid correction.
//
// One CTA owns one T x T tile of one w-plane.  It accumulates the footprints
// of every entry binned to that tile (the counting sort of rick_prep.cu lists a
// footprint that straddles tiles in each tile it touches, clipped here) into
// a shared-memory copy of the tile, then writes the whole tile once with
// coalesced 16-byte stores -- also when the tile is empty, so the planes never
// need a separate memset and HBM sees each plane byte exactly once.  No global
// atomics.  Kernel weights are evaluated in registers (separable, S per axis,
// normalised to sum 1 per axis); the fftshift checkerboard (-1)^(ju+jv) of
// the imaging transform is folded into the tap signs.
#include "rick_internal.cuh"

namespace rick {
namespace {

constexpr int kGridThreads = 256;

template <int S>
__global__ void __launch_bounds__(kGridThreads) k_grid(GridCfg c, ChunkList ch, int k0, int shift,
                                                       int accumulate, float2* __restrict__ planes)
{
    extern __shared__ float smem[];
    const int T = c.T;
    float* s_re = smem;
    float* s_im = smem + T * T;

    const int64_t tl = blockIdx.x;                 // tile within the pass
    const int kl = (int)(tl / c.ntp);              // plane within the pass
    const int rem = (int)(tl - (int64_t)kl * c.ntp);
    const int tv = rem / c.ntu, tu = rem - tv * c.ntu;
    const int64_t tg = (int64_t)(k0 + kl) * c.ntp + rem;  // global tile id
    const int u0 = tu * T, v0 = tv * T;
    const int wu = min(T, c.n - u0), wv = min(T, c.n - v0);  // ragged last tile
    float2* P = planes + (int64_t)kl * c.n * c.n;
    const int half = T >> 1;                       // float4 = 2 cells per store

    bool any = false;
    for (int q = 0; q < ch.count; ++q) any |= ch.off[q][tg + 1] != ch.off[q][tg];

    if (!any && !accumulate) {
        for (int i = threadIdx.x; i < T * half; i += kGridThreads) {
            const int row = i / half, col = (i - row * half) * 2;
            if (row < wv && col < wu)
                *reinterpret_cast<float4*>(P + (int64_t)(v0 + row) * c.n + u0 + col) =
                    make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }

    for (int i = threadIdx.x; i < T * T; i += kGridThreads) {
        float re = 0.f, im = 0.f;
        if (accumulate) {
            const int row = i / T, col = i - row * T;
            if (row < wv && col < wu) {
                const float2 x = P[(int64_t)(v0 + row) * c.n + u0 + col];
                re = x.x;
                im = x.y;
            }
        }
        s_re[i] = re;
        s_im[i] = im;
    }
    __syncthreads();

    for (int q = 0; q < ch.count; ++q) {
        const uint32_t b = ch.off[q][tg], e = ch.off[q][tg + 1];
        const float4* __restrict__ ent = ch.ent[q];
        for (uint32_t j = b + threadIdx.x; j < e; j += kGridThreads) {
            const float4 r = __ldg(ent + j);
            const int fu = first_cell(c, r.x), fv = first_cell(c, r.y);
            float gu[S], gv[S];
            eval_taps<S>(c, r.x, fu, gu);
            eval_taps<S>(c, r.y, fv, gv);
            float su = 0.f, sv = 0.f;
#pragma unroll
            for (int t = 0; t < S; ++t) {
                su += gu[t];
                sv += gv[t];
            }
            const float scale = 1.0f / (su * sv);
            float ar = r.z * scale, ai = r.w * scale;
            if (shift) {
                if ((fu + fv) & 1) {
                    ar = -ar;
                    ai = -ai;
                }
#pragma unroll
                for (int t = 1; t < S; t += 2) {
                    gu[t] = -gu[t];
                    gv[t] = -gv[t];
                }
            }
            const int lu = fu - u0, lv = fv - v0;
#pragma unroll
            for (int rr = 0; rr < S; ++rr) {
                const int row = lv + rr;
                if (row < 0 || row >= T) continue;
                const float br = ar * gv[rr], bi = ai * gv[rr];
                float* pr = s_re + row * T;
                float* pi = s_im + row * T;
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const int col = lu + t;
                    if (col < 0 || col >= T) continue;
                    atomicAdd(pr + col, br * gu[t]);
                    atomicAdd(pi + col, bi * gu[t]);
                }
            }
        }
    }
    __syncthreads();

    for (int i = threadIdx.x; i < T * half; i += kGridThreads) {
        const int row = i / half, col = (i - row * half) * 2;
        if (row < wv && col < wu) {
            const int s = row * T + col;
            *reinterpret_cast<float4*>(P + (int64_t)(v0 + row) * c.n + u0 + col) =
                make_float4(s_re[s], s_im[s], s_re[s + 1], s_im[s + 1]);
        }
    }
}

template <int S>
cudaError_t launch_grid_s(const GridCfg& c, const ChunkList& ch, int k0, int nk, bool shift,
                          bool accumulate, float2* planes, cudaStream_t s)
{
    const int64_t nblocks = (int64_t)nk * c.ntp;
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * c.T * c.T * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_grid<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_grid<S><<<(unsigned)nblocks, kGridThreads, smem, s>>>(c, ch, k0, shift ? 1 : 0, accumulate ? 1 : 0,
                                                            planes);
    return cudaGetLastError();
}

// Taper c(x) = int g(t) cos(2 pi t (x - n/2)/n) dt / int g(t) dt over
// [-S/2, S/2]: composite Simpson rule with kTaperIntervals intervals, FP64;
// the kernel samples are computed once per block into shared memory.
constexpr int kTaperIntervals = 4096;

__global__ void __launch_bounds__(256) k_taper(GridCfg c, double kparam, float* __restrict__ taper)
{
    __shared__ double g[kTaperIntervals + 1];
    const double a = -0.5 * c.S, h = (double)c.S / kTaperIntervals;
    for (int i = threadIdx.x; i <= kTaperIntervals; i += blockDim.x) {
        const double t = a + i * h;
        double val;
        if (c.kernel == RICK_KERNEL_GAUSS) {
            val = exp(-t * t / (2.0 * kparam * kparam));
        } else {
            const double z = 2.0 * t / c.S;
            val = cyl_bessel_i0(kparam * sqrt(fmax(0.0, 1.0 - z * z)));
        }
        const double wgt = (i == 0 || i == kTaperIntervals) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        g[i] = wgt * val;
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.n) return;
    const double xi2 = 2.0 * (double)(x - c.n / 2) / c.n;  // cos(2 pi t xi) = cospi(t * 2 xi)
    double num = 0.0, den = 0.0;
    for (int i = 0; i <= kTaperIntervals; ++i) {
        num += g[i] * cospi((a + i * h) * xi2);
        den += g[i];
    }
    taper[x] = (float)(num / den);
}

// Kernel value in FP64 (CUDA's exp / cyl_bessel_i0), un-normalised.
__device__ double kernel_fp64(const GridCfg& c, double kparam, double x)
{
    if (c.kernel == RICK_KERNEL_GAUSS) return exp(-x * x / (2.0 * kparam * kparam));
    const double z = 2.0 * x / c.S;
    return cyl_bessel_i0(kparam * sqrt(fmax(0.0, 1.0 - z * z)));
}

// One thread per tap t: Chebyshev interpolation of g(t + 1 - S/2 - d),
// d = (z + 1)/2, at the kPolyTerms Chebyshev nodes of z in [-1, 1], converted
// to monomial coefficients in z; values are scaled by 1/g(0) (the taps are
// normalised per axis later, so the scale cancels).  Then the binary32
// Horner evaluation is checked against FP64 on 257 points.
__global__ void k_fit_taps(GridCfg c, double kparam, float* __restrict__ coef, double* __restrict__ max_err)
{
    constexpr int D = kPolyTerms - 1;
    const int t = threadIdx.x;
    if (t >= c.S) return;
    const double pi = 3.141592653589793238462643383279502884;
    const double g0 = kernel_fp64(c, kparam, 0.0);
    double f[kPolyTerms], a[kPolyTerms];
    for (int i = 0; i <= D; ++i) {
        const double z = cos(pi * (i + 0.5) / (D + 1));
        f[i] = kernel_fp64(c, kparam, t + 1 - 0.5 * c.S - 0.5 * (z + 1.0)) / g0;
    }
    for (int k = 0; k <= D; ++k) {
        double s = 0.0;
        for (int i = 0; i <= D; ++i) s += f[i] * cos(pi * k * (i + 0.5) / (D + 1));
        a[k] = s * 2.0 / (D + 1);
    }
    a[0] *= 0.5;
    // monomial coefficients: sum_k a_k T_k(z), T_{k+1} = 2 z T_k - T_{k-1}
    double mono[kPolyTerms] = {0}, tkm1[kPolyTerms] = {0}, tk[kPolyTerms] = {0}, tn[kPolyTerms];
    tkm1[0] = 1.0;   // T_0
    tk[1] = 1.0;     // T_1
    mono[0] += a[0];
    if (D >= 1) mono[1] += a[1];
    for (int k = 1; k < D; ++k) {
        for (int j = 0; j <= D; ++j) tn[j] = (j ? 2.0 * tk[j - 1] : 0.0) - tkm1[j];
        for (int j = 0; j <= D; ++j) {
            mono[j] += a[k + 1] * tn[j];
            tkm1[j] = tk[j];
            tk[j] = tn[j];
        }
    }
    float cf[kPolyTerms];
    for (int j = 0; j <= D; ++j) {
        cf[j] = (float)mono[j];
        coef[t * kPolyTerms + j] = cf[j];
    }
    double worst = 0.0;
    for (int i = 0; i <= 256; ++i) {
        const float z = -1.0f + 2.0f * i / 256.0f;
        float v = cf[D];
        for (int j = D - 1; j >= 0; --j) v = __fmaf_rn(v, z, cf[j]);
        const double ref = kernel_fp64(c, kparam, t + 1 - 0.5 * c.S - 0.5 * ((double)z + 1.0)) / g0;
        worst = fmax(worst, fabs((double)v - ref));
    }
    max_err[t] = worst;
}

}  // namespace

cudaError_t launch_fit_taps(const GridCfg& c, double kernel_param, float* coef, double* max_err, cudaStream_t s)
{
    k_fit_taps<<<1, kMaxSupport, 0, s>>>(c, kernel_param, coef, max_err);
    return cudaGetLastError();
}

cudaError_t launch_grid(const GridCfg& c, const ChunkList& ch, int k0, int nk, bool shift_sign,
                        bool accumulate, const uint32_t* /*density*/, float2* planes, cudaStream_t s)
{
    switch (c.S) {
#define RICK_GRID_CASE(SS) \
    case SS: return launch_grid_s<SS>(c, ch, k0, nk, shift_sign, accumulate, planes, s);
        RICK_GRID_CASE(1) RICK_GRID_CASE(2) RICK_GRID_CASE(3) RICK_GRID_CASE(4)
        RICK_GRID_CASE(5) RICK_GRID_CASE(6) RICK_GRID_CASE(7) RICK_GRID_CASE(8)
        RICK_GRID_CASE(9) RICK_GRID_CASE(10) RICK_GRID_CASE(11) RICK_GRID_CASE(12)
        RICK_GRID_CASE(13) RICK_GRID_CASE(14) RICK_GRID_CASE(15) RICK_GRID_CASE(16)
#undef RICK_GRID_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_taper(const GridCfg& c, double kernel_param, float* taper, cudaStream_t s)
{
    k_taper<<<(c.n + 255) / 256, 256, 0, s>>>(c, kernel_param, taper);
    return cudaGetLastError();
}

}  // namespace rick
