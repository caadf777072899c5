// rick_taps.cu -- set-up of a handle's kernel arithmetic (once per handle):
// the degree-10 tap polynomials the gridder, the scatter and the degridder
// evaluate (fitted in FP64 on the device), and the taper c(x) that grid
// correction divides the image by (the normalised Fourier transform of the
// continuous kernel, by FP64 quadrature).
#include "rick_internal.cuh"

namespace rick {
namespace {

// Taper c(x) = int g(t) cos(2 pi t (x - n/2)/n) dt / int g(t) dt over
// [-S/2, S/2]: composite Simpson rule with kTaperIntervals intervals, FP64;
// the weighted kernel samples are computed once (k_taper_samples), then one
// CTA per pixel sums the rule.
constexpr int kTaperIntervals = 4096;

// Simpson-weighted kernel samples w_i g(t_i), t_i = -S/2 + i S / kTaperIntervals.
__global__ void k_taper_samples(GridCfg c, double kparam, double* __restrict__ g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kTaperIntervals) return;
    const double a = -0.5 * c.S, h = (double)c.S / kTaperIntervals;
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

// One CTA per pixel x: its threads split the quadrature sum, then reduce.
constexpr int kTaperThreads = 128;

__global__ void __launch_bounds__(kTaperThreads) k_taper(GridCfg c, const double* __restrict__ g,
                                                         float* __restrict__ taper)
{
    const int x = blockIdx.x;
    const double a = -0.5 * c.S, h = (double)c.S / kTaperIntervals;
    const double xi2 = 2.0 * (double)(x - c.n / 2) / c.n;  // cos(2 pi t xi) = cospi(t * 2 xi)
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i <= kTaperIntervals; i += kTaperThreads) {
        num += g[i] * cospi((a + i * h) * xi2);
        den += g[i];
    }
    __shared__ double sn[kTaperThreads / 32], sd[kTaperThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sn[threadIdx.x >> 5] = num;
        sd[threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0.0, td = 0.0;
        for (int k = 0; k < kTaperThreads / 32; ++k) {
            tn += sn[k];
            td += sd[k];
        }
        taper[x] = (float)(tn / td);
    }
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

// Grid correction in w (w-support Sw > 1): hw(xi) = int h(x) cos(2 pi x xi)
// dx / int h over [-Sw/2, Sw/2], h the kernel family with support Sw, at
// xi_j = xi_max j / (len - 1); FP64 Simpson rule like the taper.
__global__ void k_w_samples(GridCfg c, double* __restrict__ g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kTaperIntervals) return;
    const double a = -0.5 * c.Sw, h = (double)c.Sw / kTaperIntervals;
    const double t = a + i * h;
    double val;
    if (c.kernel == RICK_KERNEL_GAUSS) {
        const double sig = c.Sw / 6.0;
        val = exp(-t * t / (2.0 * sig * sig));
    } else {
        const double z = 2.0 * t / c.Sw;
        val = cyl_bessel_i0(2.34 * c.Sw * sqrt(fmax(0.0, 1.0 - z * z)));
    }
    const double wgt = (i == 0 || i == kTaperIntervals) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    g[i] = wgt * val;
}

__global__ void __launch_bounds__(kTaperThreads) k_wcorr(GridCfg c, const double* __restrict__ g, double xi_max,
                                                         int len, float* __restrict__ out)
{
    const int j = blockIdx.x;
    const double a = -0.5 * c.Sw, h = (double)c.Sw / kTaperIntervals;
    const double xi2 = 2.0 * xi_max * j / (len - 1);  // cos(2 pi x xi) = cospi(x * 2 xi)
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i <= kTaperIntervals; i += kTaperThreads) {
        num += g[i] * cospi((a + i * h) * xi2);
        den += g[i];
    }
    __shared__ double sn[kTaperThreads / 32], sd[kTaperThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sn[threadIdx.x >> 5] = num;
        sd[threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0.0, td = 0.0;
        for (int k = 0; k < kTaperThreads / 32; ++k) {
            tn += sn[k];
            td += sd[k];
        }
        out[j] = (float)(tn / td);
    }
}

}  // namespace

cudaError_t launch_wcorr(const GridCfg& c, double xi_max, int len, float* out, cudaStream_t s)
{
    double* g = nullptr;
    cudaError_t e = cudaMalloc((void**)&g, sizeof(double) * (kTaperIntervals + 1));
    if (e != cudaSuccess) return e;
    k_w_samples<<<(kTaperIntervals + 256) / 256, 256, 0, s>>>(c, g);
    k_wcorr<<<len, kTaperThreads, 0, s>>>(c, g, xi_max, len, out);
    e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(g);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_fit_taps(const GridCfg& c, double kernel_param, float* coef, double* max_err, cudaStream_t s)
{
    k_fit_taps<<<1, kMaxSupport, 0, s>>>(c, kernel_param, coef, max_err);
    return cudaGetLastError();
}

cudaError_t launch_taper(const GridCfg& c, double kernel_param, float* taper, cudaStream_t s)
{
    double* g = nullptr;
    cudaError_t e = cudaMalloc((void**)&g, sizeof(double) * (kTaperIntervals + 1));
    if (e != cudaSuccess) return e;
    k_taper_samples<<<(kTaperIntervals + 256) / 256, 256, 0, s>>>(c, kernel_param, g);
    k_taper<<<c.n, kTaperThreads, 0, s>>>(c, g, taper);
    e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(g);
    return e != cudaSuccess ? e : e2;
}

}  // namespace rick
