// rick_stack.cu -- step 4 of the workflow (Sec. 2.1): w-term correction and
// reduction of the w-planes into one image, Eq. 1:
//     I(l, m) = sum_k P_k(l, m) exp(+2 pi i w_k (n - 1)),
// fused with the fftshift sign of the plane transform and with the final
// normalisation (1 / sum of weights, optional taper division and factor n).
//
// One thread owns two adjacent pixels; it streams the group's planes once
// (16-byte loads, evict-first), accumulates in registers and writes the image
// once per group.  Accuracy: n - 1 and w_k (n - 1) are carried as float pairs
// (hi + lo, error-free products), so the phase in turns is exact to ~1e-7
// even when |w (n - 1)| reaches hundreds of turns; the screen is advanced by a
// complex rotation per plane and re-evaluated directly every kResync planes.
#include "rick_internal.cuh"

namespace rick {
namespace {

constexpr int kStackThreads = 256;
constexpr int kResync = 8;

struct FF {
    float hi, lo;
};

// a * b for float pairs, lo terms to first order.
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float p = a.hi * b.hi;
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return FF{p, e + __fmaf_rn(a.hi, b.lo, a.lo * b.hi)};
}

// exp(2 pi i (hi + lo)) with the integer part of hi removed exactly.
__device__ __forceinline__ float2 turns_to_phasor(float hi, float lo)
{
    const float f = (hi - rintf(hi)) + lo;
    float s, c;
    sincospif(2.0f * f, &s, &c);
    return make_float2(c, s);
}

// Phase in turns of plane k: A + k B, A = wb (n-1), B = dw (n-1).
__device__ __forceinline__ float2 screen(FF A, FF B, int k)
{
    const float kf = (float)k;
    const float kb = kf * B.hi;
    const float kbe = __fmaf_rn(kf, B.hi, -kb);
    const float s = A.hi + kb;                 // two-sum of A.hi + kb
    const float bb = s - A.hi;
    const float err = (A.hi - (s - bb)) + (kb - bb);
    return turns_to_phasor(s, err + kbe + A.lo + kf * B.lo);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct PixelScreen {
    FF A, B;
    float nm1;
    bool sky;
};

__device__ __forceinline__ PixelScreen pixel_screen(const StackArgs& a, int x, int y)
{
    PixelScreen ps;
    const int ix = x - a.n / 2, iy = y - a.n / 2;
    const int q = ix * ix + iy * iy;                        // exact integer
    const float qh = (float)q;
    const float ql = (float)(q - (int)qh);
    const FF r2 = ff_mul(FF{qh, ql}, FF{a.dl2_hi, a.dl2_lo});  // l^2 + m^2
    ps.sky = r2.hi < 1.0f;
    // n - 1 = -r2 / (2 + (n - 1)); eps is a binary32 first guess of n - 1
    const float eps = ps.sky ? -r2.hi / (1.0f + sqrtf(1.0f - r2.hi)) : 0.0f;
    const float he = 0.5f * eps;
    FF nm1;
    nm1.hi = -0.5f * r2.hi;
    nm1.lo = -0.5f * r2.lo + (0.5f * r2.hi) * (he / (1.0f + he));
    ps.nm1 = nm1.hi + nm1.lo;
    ps.A = ff_mul(FF{a.wb_hi, a.wb_lo}, nm1);
    ps.B = ff_mul(FF{a.dw_hi, a.dw_lo}, nm1);
    return ps;
}

__global__ void __launch_bounds__(kStackThreads) k_stack(StackArgs a, const float2* __restrict__ planes,
                                                         float2* __restrict__ acc,
                                                         const float* __restrict__ taper,
                                                         const double* __restrict__ sum_w, void* image)
{
    const int halfn = a.n >> 1;
    const int64_t idx = blockIdx.x * (int64_t)kStackThreads + threadIdx.x;
    if (idx >= (int64_t)a.n * halfn) return;
    const int y = (int)(idx / halfn);
    const int x0 = (int)(idx - (int64_t)y * halfn) * 2;
    const int64_t pix = (int64_t)y * a.n + x0;
    const int64_t nn = (int64_t)a.n * a.n;

    PixelScreen s0 = pixel_screen(a, x0, y), s1 = pixel_screen(a, x0 + 1, y);
    const float2 rho0 = turns_to_phasor(s0.B.hi, s0.B.lo);
    const float2 rho1 = turns_to_phasor(s1.B.hi, s1.B.lo);
    float2 z0 = make_float2(1.f, 0.f), z1 = z0;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;

    const float4* p = reinterpret_cast<const float4*>(planes + pix);
    const int64_t stride4 = nn >> 1;  // plane stride in float4
#pragma unroll 4
    for (int kl = 0; kl < a.nk; ++kl) {
        const float4 v = __ldcs(p + kl * stride4);
        if (kl % kResync == 0) {
            z0 = screen(s0.A, s0.B, a.k0 + kl);
            z1 = screen(s1.A, s1.B, a.k0 + kl);
        } else {
            z0 = cmul(z0, rho0);
            z1 = cmul(z1, rho1);
        }
        const float2 c0 = cmul(make_float2(v.x, v.y), z0);
        const float2 c1 = cmul(make_float2(v.z, v.w), z1);
        a0.x += c0.x;
        a0.y += c0.y;
        a1.x += c1.x;
        a1.y += c1.y;
    }
    // fftshift sign (-1)^(x + y); x0 even so the second pixel has the opposite sign
    if (y & 1) {
        a0 = make_float2(-a0.x, -a0.y);
    } else {
        a1 = make_float2(-a1.x, -a1.y);
    }
    if (!s0.sky) a0 = make_float2(0.f, 0.f);
    if (!s1.sky) a1 = make_float2(0.f, 0.f);
    if (!a.first) {
        const float4 prev = *reinterpret_cast<const float4*>(acc + pix);
        a0.x += prev.x;
        a0.y += prev.y;
        a1.x += prev.z;
        a1.y += prev.w;
    }
    if (!a.last) {
        *reinterpret_cast<float4*>(acc + pix) = make_float4(a0.x, a0.y, a1.x, a1.y);
        return;
    }
    const double sw = *sum_w;
    const float inv_sw = (sw != 0.0) ? (float)(1.0 / sw) : 0.0f;
    float f0 = inv_sw, f1 = inv_sw;
    if (a.flags & RICK_GRID_CORRECT) {
        const float ty = __ldg(taper + y);
        f0 = f0 / (__ldg(taper + x0) * ty);
        f1 = f1 / (__ldg(taper + x0 + 1) * ty);
    }
    if (a.flags & RICK_APPLY_N) {
        f0 *= 1.0f + s0.nm1;
        f1 *= 1.0f + s1.nm1;
    }
    if (a.wcorr) {  // grid correction in w (w-support > 1)
        f0 /= wcorr_at(a, s0.nm1);
        f1 /= wcorr_at(a, s1.nm1);
    }
    if (a.flags & RICK_REAL_IMAGE) {
        reinterpret_cast<float2*>(image)[pix >> 1] = make_float2(a0.x * f0, a1.x * f1);
    } else {
        reinterpret_cast<float4*>(image)[pix >> 1] = make_float4(a0.x * f0, a0.y * f0, a1.x * f1, a1.y * f1);
    }
}

// Adjoint of k_stack (and of the finalisation): from an image gradient r,
// write for every plane k of the group  Q_k = s(x,y) * R * exp(-2 pi i w_k (n-1)),
// R = r / sum_w / taper(x) taper(y) * n  (per flags), ready for a forward FFT.
__global__ void __launch_bounds__(kStackThreads) k_spread(StackArgs a, const void* __restrict__ rimg,
                                                          const float* __restrict__ taper,
                                                          const double* __restrict__ sum_w,
                                                          float2* __restrict__ planes)
{
    const int halfn = a.n >> 1;
    const int64_t idx = blockIdx.x * (int64_t)kStackThreads + threadIdx.x;
    if (idx >= (int64_t)a.n * halfn) return;
    const int y = (int)(idx / halfn);
    const int x0 = (int)(idx - (int64_t)y * halfn) * 2;
    const int64_t pix = (int64_t)y * a.n + x0;
    const int64_t nn = (int64_t)a.n * a.n;

    PixelScreen s0 = pixel_screen(a, x0, y), s1 = pixel_screen(a, x0 + 1, y);
    float2 r0, r1;
    if (a.flags & RICK_REAL_IMAGE) {
        const float2 rr = reinterpret_cast<const float2*>(rimg)[pix >> 1];
        r0 = make_float2(rr.x, 0.f);
        r1 = make_float2(rr.y, 0.f);
    } else {
        const float4 rr = reinterpret_cast<const float4*>(rimg)[pix >> 1];
        r0 = make_float2(rr.x, rr.y);
        r1 = make_float2(rr.z, rr.w);
    }
    const double sw = *sum_w;
    const float inv_sw = (sw != 0.0) ? (float)(1.0 / sw) : 0.0f;
    float f0 = inv_sw, f1 = inv_sw;
    if (a.flags & RICK_GRID_CORRECT) {
        const float ty = __ldg(taper + y);
        f0 = f0 / (__ldg(taper + x0) * ty);
        f1 = f1 / (__ldg(taper + x0 + 1) * ty);
    }
    if (a.flags & RICK_APPLY_N) {
        f0 *= 1.0f + s0.nm1;
        f1 *= 1.0f + s1.nm1;
    }
    if (a.wcorr) {  // grid correction in w (w-support > 1)
        f0 /= wcorr_at(a, s0.nm1);
        f1 /= wcorr_at(a, s1.nm1);
    }
    // fftshift sign (-1)^(x + y) and the sky mask
    if (y & 1) f0 = -f0; else f1 = -f1;
    if (!s0.sky) f0 = 0.f;
    if (!s1.sky) f1 = 0.f;
    r0 = make_float2(r0.x * f0, r0.y * f0);
    r1 = make_float2(r1.x * f1, r1.y * f1);

    const float2 rho0 = turns_to_phasor(s0.B.hi, s0.B.lo);
    const float2 rho1 = turns_to_phasor(s1.B.hi, s1.B.lo);
    float2 z0 = make_float2(1.f, 0.f), z1 = z0;
    float4* p = reinterpret_cast<float4*>(planes + pix);
    const int64_t stride4 = nn >> 1;
    for (int kl = 0; kl < a.nk; ++kl) {
        if (kl % kResync == 0) {
            z0 = screen(s0.A, s0.B, a.k0 + kl);
            z1 = screen(s1.A, s1.B, a.k0 + kl);
        } else {
            z0 = cmul(z0, rho0);
            z1 = cmul(z1, rho1);
        }
        // multiply by conj(z)
        const float2 c0 = make_float2(r0.x * z0.x + r0.y * z0.y, r0.y * z0.x - r0.x * z0.y);
        const float2 c1 = make_float2(r1.x * z1.x + r1.y * z1.y, r1.y * z1.x - r1.x * z1.y);
        __stcs(p + kl * stride4, make_float4(c0.x, c0.y, c1.x, c1.y));
    }
}

}  // namespace

cudaError_t launch_spread(const StackArgs& a, const void* rimg, const float* taper, const double* sum_w,
                          float2* planes, cudaStream_t s)
{
    const int64_t threads = (int64_t)a.n * (a.n / 2);
    const int64_t blocks = (threads + kStackThreads - 1) / kStackThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_spread<<<(unsigned)blocks, kStackThreads, 0, s>>>(a, rimg, taper, sum_w, planes);
    return cudaGetLastError();
}

cudaError_t launch_stack(const StackArgs& a, const float2* planes, float2* acc, const float* taper,
                         const double* sum_w, void* image, cudaStream_t s)
{
    const int64_t threads = (int64_t)a.n * (a.n / 2);
    const int64_t blocks = (threads + kStackThreads - 1) / kStackThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_stack<<<(unsigned)blocks, kStackThreads, 0, s>>>(a, planes, acc, taper, sum_w, image);
    return cudaGetLastError();
}

}  // namespace rick
