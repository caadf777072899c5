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
#include "rick_tma.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

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
    // n <= 32768: idx < n * n / 2 <= 2^29, so 32-bit division is exact
    const uint32_t ui = (uint32_t)idx;
    const int y = (int)(ui / (uint32_t)halfn);
    const int x0 = (int)(ui - (uint32_t)y * (uint32_t)halfn) * 2;
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
    // n <= 32768: idx < n * n / 2 <= 2^29, so 32-bit division is exact
    const uint32_t ui = (uint32_t)idx;
    const int y = (int)(ui / (uint32_t)halfn);
    const int x0 = (int)(ui - (uint32_t)y * (uint32_t)halfn) * 2;
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

// ---------------------------------------------------------------------------
// Column transform + w-screen + plane stack in one pass (the split transform
// of power-of-two n in [64, 16384]).  cuFFT has already transformed the rows
// and k_colfft the first factor of the column dimension: with n = N1 * N2
// (N2 = 16), row v = N2 a + b and output row y = f1 + N1 f2 (w_M =
// exp(2 pi i / M), the inverse sign),
//     Y[N2 f1 + b] = sum_a x[N2 a + b] w_N1^(a f1)
// is in the plane, and the remaining factor
//     X[f1 + N1 f2] = sum_b w_N2^(b f2) (w_n^(b f1) Y[N2 f1 + b])
// is a 16-point transform of the 16 rows N2 f1 + b, b = 0 .. 15, per f1 (in
// the planes' b-major row order, memory rows b N1 + f1: 16 rows N1 apart).
// A CTA owns one f1 and 32 columns.  It streams those rows of every plane of
// the group through a ring of shared-memory stages, one 3D TMA box per plane
// completing on the stage's mbarrier, does the 16 = 4 x 4 transform in two
// register passes with an exchange inside each warp (b = 4 b1 + b0,
// f2 = g0 + 4 g1: w_16^(b f2) = w_4^(b1 g0) w_16^(b0 g0) w_4^(b0 g1)), and sums
// the planes with their w-screen per pixel.  The planes are read once and
// never written back.

constexpr int kColQ = 4;                     // N2 = kColQ^2 = 16-point column factor
constexpr int kColN2 = kColQ * kColQ;
constexpr int kColW = 32;                    // columns per CTA: one 256-byte row segment
constexpr int kColWarps = kColW / 8;         // a warp owns 8 columns x kColQ values of j
constexpr int kColThreads = 32 * kColWarps;
constexpr int kColStages = 5;  // 35.7 KB per CTA with the screens: six CTAs per SM
constexpr int kColPitch = kColW;             // complex values per staged row (the TMA box, dense)
// lanes: column cl = lane % 8 of the warp's 8, j = lane / 8; a half warp then
// reads two rows of 8 columns of a stage (2-way bank conflict, the dense TMA
// rows being 256 bytes apart) and, with this exchange pitch (two rows 320
// bytes apart: 16 banks), writes and reads the exchange without conflicts
constexpr int kColExPitch = 40;              // complex values per g of a warp's exchange
constexpr size_t kColStageBytes = (size_t)kColN2 * kColPitch * sizeof(float2);
constexpr size_t kColExBytes = (size_t)kColWarps * kColQ * kColExPitch * sizeof(float2);
// each thread's 4 pixels: the screen's phase coefficients (A.hi, A.lo, B.hi,
// B.lo) and n - 1, evaluated once per block
constexpr size_t kColScrBytes = (size_t)kColQ * kColThreads * (sizeof(float4) + sizeof(float));
// stages (TMA destinations, at the 128-byte aligned start) | full and empty
// mbarriers | the warps' exchange buffers | pixel screens | abort flag and issue count
constexpr size_t kColSmem = kColStages * kColStageBytes + 2 * kColStages * sizeof(unsigned long long) + kColExBytes +
                            kColScrBytes + 2 * sizeof(int);
constexpr unsigned long long kColWaitNs = 1000000000ull;  // default bound of one wait: 1 s
// planes summed by Horner's rule between direct evaluations of the screen
// (the rotation per plane is applied in binary32, relative error ~1e-7 each)
constexpr int kColResync = 32;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// In-place 4-point DFT with the + sign, natural order in and out.
__device__ __forceinline__ void dft4(float2 (&v)[4])
{
    const float2 a0 = cadd(v[0], v[2]), a2 = csub(v[0], v[2]);
    const float2 a1 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const float2 a3 = make_float2(-d.y, d.x);  // times +i
    v[0] = cadd(a0, a1);
    v[2] = csub(a0, a1);
    v[1] = cadd(a2, a3);
    v[3] = csub(a2, a3);
}

// planes: the group's nk planes, rows and the first column factor already
// transformed; grid (n / kColW, N1).  Warp w owns columns x0 + 8 w + cl
// (cl < 8) and lane j + 4 cl: b0 = j in the first pass, g0 = j in the second,
// so the exchange between the passes stays inside the warp.  Stage s has a
// "full" mbarrier (the bulk copies) and an "empty" one (one arrival per warp
// once it has read the stage); warp 0 refills a stage when it is empty.
// Planes are taken from the last to the first and summed per pixel by
// Horner's rule, h <- h rho + v, times the screen of the block's first plane.
// err: set to 1 when a bounded wait ran out.
__global__ void __launch_bounds__(kColThreads, 6) k_colstack(const __grid_constant__ CUtensorMap map,
                                                             StackArgs a_in, int n1, float2* __restrict__ acc,
                                                             const float* __restrict__ taper,
                                                             const double* __restrict__ sum_w, void* image,
                                                             unsigned long long* err)
{
    // the launch's channel (batched imaging: one launch over the channels of
    // a plane group) or the single image
    StackArgs a = a_in;
    if (a_in.chan_screen) {
        const int ch = a_in.chan0 + (int)blockIdx.z;
        const float4 cs = __ldg(a_in.chan_screen + ch);
        a.wb_hi = cs.x;
        a.wb_lo = cs.y;
        a.dw_hi = cs.z;
        a.dw_lo = cs.w;
        a.plane0 = a_in.plane0 + (int)blockIdx.z * a_in.nk;
        sum_w += ch;
        image = reinterpret_cast<float*>(image) + (size_t)ch * a_in.img_stride;
    }
    extern __shared__ __align__(128) unsigned char col_smem[];
    float2* stage = reinterpret_cast<float2*>(col_smem);  // [stages][N2][kColPitch]
    unsigned long long* full = reinterpret_cast<unsigned long long*>(col_smem + kColStages * kColStageBytes);
    unsigned long long* empty = full + kColStages;
    float2* exw = reinterpret_cast<float2*>(col_smem + kColStages * kColStageBytes +
                                            2 * kColStages * sizeof(unsigned long long));
    float4* scr = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(exw) + kColExBytes);  // [g][t]
    float* snm1 = reinterpret_cast<float*>(scr + kColQ * kColThreads);                              // [g][t]
    int& s_abort = *reinterpret_cast<int*>(snm1 + kColQ * kColThreads);
    int& s_issued = (&s_abort)[1];

    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int cl = lane & 7, j = lane >> 3;
    const int cw = 8 * w + cl;  // column in the CTA's strip
    const int n = a.n, nk = a.nk;
    const int x0 = blockIdx.x * kColW, x = x0 + cw;
    const int f1 = blockIdx.y;
    float2* ex = exw + (size_t)w * kColQ * kColExPitch;
    const unsigned long long limit = a.wait_ns ? a.wait_ns : kColWaitNs;

    if (t == 0) {
        s_abort = 0;
        for (int st = 0; st < kColStages; ++st) {
            mbar_init(smem_u32(full + st), 1);
            mbar_init(smem_u32(empty + st), kColWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // slot i of the pipeline carries plane nk - 1 - i into stage i % stages:
    // one TMA box of kColW columns x N2 rows (b = 0 .. 15) at (x0, f1,
    // 16 plane) of the map's [16 planes][N1][n] view of the plane buffer
    auto issue = [&](int i) {  // called by all of warp 0
        if (lane == 0 && i + 1 != a.skip_slot1) {
            const int st = i % kColStages;
            const uint32_t bar = smem_u32(full + st);
            mbar_expect(bar, (uint32_t)kColStageBytes);
            tma_load_3d(smem_u32(stage + (size_t)st * kColN2 * kColPitch), &map, x0, f1,
                        (a.plane0 + nk - 1 - i) * kColN2, bar);
        }
        __syncwarp();
    };
    int issued = nk < kColStages ? nk : kColStages;
    if (w == 0)
        for (int i = 0; i < issued; ++i) issue(i);

    // twiddles: w_n^(b f1) for the thread's rows b = 4 b1 + j, and w_16^(j g0),
    // each a power series of one exactly evaluated step (integer phases mod n)
    float2 tw[kColQ], tin[kColQ];
    {
        float sn, cs;
        sincospif(2.0f * (float)((int)(((int64_t)j * f1) % n)) / (float)n, &sn, &cs);
        tw[0] = make_float2(cs, sn);
        sincospif(2.0f * (float)((int)(((int64_t)kColQ * f1) % n)) / (float)n, &sn, &cs);
        const float2 step = make_float2(cs, sn);
        sincospif(2.0f * (float)j / (float)kColN2, &sn, &cs);
        const float2 istep = make_float2(cs, sn);
        tin[0] = make_float2(1.f, 0.f);
#pragma unroll
        for (int q = 1; q < kColQ; ++q) {
            tw[q] = cmul(tw[q - 1], step);
            tin[q] = cmul(tin[q - 1], istep);
        }
    }

    // the thread's output pixels (x, y_g), y_g = f1 + N1 (j + 4 g): the screen's
    // rotation per plane, the Horner sum of the current block and the total
    float2 rho[kColQ], h[kColQ], sum[kColQ];
    unsigned sky = 0;
#pragma unroll
    for (int g = 0; g < kColQ; ++g) {
        const PixelScreen ps = pixel_screen(a, x, f1 + n1 * (j + kColQ * g));
        scr[g * kColThreads + t] = make_float4(ps.A.hi, ps.A.lo, ps.B.hi, ps.B.lo);
        snm1[g * kColThreads + t] = ps.nm1;
        sky |= (ps.sky ? 1u : 0u) << g;
        rho[g] = turns_to_phasor(ps.B.hi, ps.B.lo);
        h[g] = make_float2(0.f, 0.f);
        sum[g] = make_float2(0.f, 0.f);
    }

    bool ok = true;
    // two planes per trip (measured: 1.115 -> 1.082 ms at 4096^2 x 32; four: 1.158)
#pragma unroll 2
    for (int i = 0; i < nk && ok; ++i) {
        const int st = i % kColStages;
        const uint32_t ph = (uint32_t)((i / kColStages) & 1);
        // one decision per warp: a lane whose wait ran out takes its warp out
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(full + st), ph, &s_abort, limit));
        // first pass: 4-point transforms over b1 of w_n^(b f1) Y[b], times w_16^(b0 g0)
        float2 v[kColQ];
        const float2* blk = stage + (size_t)st * kColN2 * kColPitch;
#pragma unroll
        for (int q = 0; q < kColQ; ++q) v[q] = cmul(blk[(kColQ * q + j) * kColPitch + cw], tw[q]);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(empty + st));  // this warp is done with the stage
        dft4(v);
        ex[8 * j + cl] = v[0];  // w_16^0 = 1
#pragma unroll
        for (int g = 1; g < kColQ; ++g) ex[g * kColExPitch + 8 * j + cl] = cmul(v[g], tin[g]);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kColQ; ++q) v[q] = ex[j * kColExPitch + 8 * q + cl];
        __syncwarp();
        // second pass: 4-point transforms over b0 for g0 = j
        dft4(v);
        // Horner step of plane p; at a block start, times the screen of plane p
        const int p = nk - 1 - i;
#pragma unroll
        for (int g = 0; g < kColQ; ++g) h[g] = cadd(cmul(h[g], rho[g]), v[g]);
        if (p % kColResync == 0) {
#pragma unroll
            for (int g = 0; g < kColQ; ++g) {
                const float4 ab = scr[g * kColThreads + t];
                const float2 r = cmul(h[g], screen(FF{ab.x, ab.y}, FF{ab.z, ab.w}, a.k0 + p));
                sum[g] = cadd(sum[g], r);
                h[g] = make_float2(0.f, 0.f);
            }
        }
        // warp 0 refills the stage once every warp has read it
        if (w == 0 && ok && i + kColStages < nk) {
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(empty + st), ph, &s_abort, limit));
            if (ok) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(i + kColStages);
                ++issued;
            }
        }
        if (!ok) s_abort = 1;
    }
    if (w == 0 && lane == 0) s_issued = issued;
    __syncthreads();
    if (s_abort) {
        // leave no bulk copy in flight into this CTA's shared memory: wait
        // (bounded) for the last slot issued into every stage, in slot order
        if (t == 0) {
            atomicOr(err, 1ull);
            const int last = s_issued;
            for (int i = last > kColStages ? last - kColStages : 0; i < last; ++i) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try(smem_u32(full + i % kColStages), (uint32_t)((i / kColStages) & 1)) &&
                       global_ns() - t0 <= limit) {
                }
            }
        }
        __syncthreads();
        return;
    }

    const double sw = *sum_w;
    const float inv_sw = (sw != 0.0) ? (float)(1.0 / sw) : 0.0f;
#pragma unroll
    for (int g = 0; g < kColQ; ++g) {
        const int y = f1 + n1 * (j + kColQ * g);
        const int64_t pix = (int64_t)y * n + x;
        float2 r = sum[g];
        if ((x + y) & 1) r = make_float2(-r.x, -r.y);  // fftshift sign (-1)^(x + y)
        if (!((sky >> g) & 1u)) r = make_float2(0.f, 0.f);
        const float nm1 = snm1[g * kColThreads + t];
        if (!a.first) {
            const float2 prev = acc[pix];
            r.x += prev.x;
            r.y += prev.y;
        }
        if (!a.last) {
            acc[pix] = r;
            continue;
        }
        float f = inv_sw;
        if (a.flags & RICK_GRID_CORRECT) f = f / (__ldg(taper + x) * __ldg(taper + y));
        if (a.flags & RICK_APPLY_N) f *= 1.0f + nm1;
        if (a.wcorr) f /= wcorr_at(a, nm1);
        if (a.flags & RICK_REAL_IMAGE)
            reinterpret_cast<float*>(image)[pix] = r.x * f;
        else
            reinterpret_cast<float2*>(image)[pix] = make_float2(r.x * f, r.y * f);
    }
}
// In-place 4-point DFT with the - sign (the adjoint of dft4 up to order).
__device__ __forceinline__ void dft4m(float2 (&v)[4])
{
    const float2 a0 = cadd(v[0], v[2]), a2 = csub(v[0], v[2]);
    const float2 a1 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const float2 a3 = make_float2(d.y, -d.x);  // times -i
    v[0] = cadd(a0, a1);
    v[2] = csub(a0, a1);
    v[1] = cadd(a2, a3);
    v[3] = csub(a2, a3);
}

__device__ __forceinline__ float2 cmulc(float2 a, float2 b)  // a * conj(b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Adjoint of k_colstack (the backward pass of imaging and prediction, n with
// the split transform): for one f1 and 32 columns, every plane k of the group
// gets the rows 16 f1 + b (memory rows b N1 + f1, the b-major order)
//     Y'[16 f1 + b] = conj(w_n^(b f1)) sum_f2 w_16^(-b f2) Z_k[f1 + N1 f2],
//     Z_k(x, y) = R(x, y) conj(screen_k(x, y)),
// R the adjoint of the finalisation applied to the image gradient (sign,
// sky mask, 1 / weight sum, taper, n and w correction per flags, as
// k_spread).  cuFFT then applies the forward N1-point column factor and the
// forward row transform: together the 2D forward transform of the screened
// planes.  The thread's pixels, twiddles and the warp-local exchange are
// those of k_colstack, the two 4-point passes taken in reverse order with
// the conjugate sign; nothing waits on memory but the stores.
__global__ void __launch_bounds__(kColThreads, 5) k_spreadcol(StackArgs a, int n1, const void* __restrict__ rimg,
                                                              const float* __restrict__ taper,
                                                              const double* __restrict__ sum_w,
                                                              float2* __restrict__ planes)
{
    __shared__ float2 exw[kColWarps * kColQ * kColExPitch];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int j = lane & (kColQ - 1), cl = lane >> 2;
    const int n = a.n;
    const int x = blockIdx.x * kColW + 8 * w + cl;
    const int f1 = blockIdx.y;
    const int64_t nn = (int64_t)n * n;
    float2* ex = exw + (size_t)w * kColQ * kColExPitch;

    float2 tw[kColQ], tin[kColQ];
    {
        float sn, cs;
        sincospif(2.0f * (float)((int)(((int64_t)j * f1) % n)) / (float)n, &sn, &cs);
        tw[0] = make_float2(cs, sn);
        sincospif(2.0f * (float)((int)(((int64_t)kColQ * f1) % n)) / (float)n, &sn, &cs);
        const float2 step = make_float2(cs, sn);
        sincospif(2.0f * (float)j / (float)kColN2, &sn, &cs);
        const float2 istep = make_float2(cs, sn);
        tin[0] = make_float2(1.f, 0.f);
#pragma unroll
        for (int q = 1; q < kColQ; ++q) {
            tw[q] = cmul(tw[q - 1], step);
            tin[q] = cmul(tin[q - 1], istep);
        }
    }

    // the thread's pixels (x, y_g), y_g = f1 + N1 (j + 4 g): R, the screen's
    // rotation per plane and the screen of the current plane
    const double sw = *sum_w;
    const float inv_sw = (sw != 0.0) ? (float)(1.0 / sw) : 0.0f;
    float2 r[kColQ], rho[kColQ], z[kColQ];
#pragma unroll
    for (int g = 0; g < kColQ; ++g) {
        const int y = f1 + n1 * (j + kColQ * g);
        const int64_t pix = (int64_t)y * n + x;
        const PixelScreen ps = pixel_screen(a, x, y);
        float2 rv = (a.flags & RICK_REAL_IMAGE) ? make_float2(reinterpret_cast<const float*>(rimg)[pix], 0.f)
                                                : reinterpret_cast<const float2*>(rimg)[pix];
        float f = inv_sw;
        if (a.flags & RICK_GRID_CORRECT) f = f / (__ldg(taper + x) * __ldg(taper + y));
        if (a.flags & RICK_APPLY_N) f *= 1.0f + ps.nm1;
        if (a.wcorr) f /= wcorr_at(a, ps.nm1);
        if ((x + y) & 1) f = -f;  // fftshift sign (-1)^(x + y)
        if (!ps.sky) f = 0.f;
        r[g] = make_float2(rv.x * f, rv.y * f);
        rho[g] = turns_to_phasor(ps.B.hi, ps.B.lo);
        z[g] = screen(ps.A, ps.B, a.k0);
    }

    // grid row 16 f1 + b (b = j + 4 q) is memory row b N1 + f1
    const int64_t row0 = f1, bstride = (int64_t)n1 * n;
#pragma unroll 2
    for (int p = 0; p < a.nk; ++p) {
        float2 v[kColQ];
#pragma unroll
        for (int g = 0; g < kColQ; ++g) {
            if (p > 0) {
                if (p % kColResync == 0) {
                    const PixelScreen ps = pixel_screen(a, x, f1 + n1 * (j + kColQ * g));
                    z[g] = screen(ps.A, ps.B, a.k0 + p);
                } else {
                    z[g] = cmul(z[g], rho[g]);
                }
            }
            v[g] = cmulc(r[g], z[g]);
        }
        // over g1 -> b0 (this thread is g0 = j), times conj(w_16^(b0 g0))
        dft4m(v);
        ex[8 * j + cl] = v[0];
#pragma unroll
        for (int q = 1; q < kColQ; ++q) ex[q * kColExPitch + 8 * j + cl] = cmulc(v[q], tin[q]);
        __syncwarp();
        // over g0 -> b1 (this thread is b0 = j), times conj(w_n^(b f1))
#pragma unroll
        for (int q = 0; q < kColQ; ++q) v[q] = ex[j * kColExPitch + 8 * q + cl];
        __syncwarp();
        dft4m(v);
        float2* dst = planes + (int64_t)p * nn + (row0 + (int64_t)j * n1) * n + x;
#pragma unroll
        for (int q = 0; q < kColQ; ++q) __stcs(dst + kColQ * q * bstride, cmulc(v[q], tw[q]));
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


cudaError_t launch_spreadcol(const StackArgs& a, int n1, int n2, const void* rimg, const float* taper,
                             const double* sum_w, float2* planes, cudaStream_t s)
{
    if (a.nk <= 0) return cudaSuccess;
    if (n2 != kColN2 || (int64_t)n1 * n2 != a.n || a.n % kColW != 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(a.n / kColW), (unsigned)n1);
    k_spreadcol<<<grid, kColThreads, 0, s>>>(a, n1, rimg, taper, sum_w, planes);
    return cudaGetLastError();
}

bool colstack_shape(int n, int* n1, int* n2)
{
    if (n < 64 || n > 16384 || (n & (n - 1))) return false;
    *n2 = kColN2;
    *n1 = n / kColN2;
    return true;
}

cudaError_t encode_colstack_map(void* map, const float2* planes, int n, int planes_in_buffer)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        const cudaError_t e =
            cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    // the plane buffer as [planes_in_buffer * 16][N1][n] 8-byte complex
    // values (b-major rows: grid row 16 f1 + b of plane p is (f1, 16 p + b));
    // a box is kColW columns of one f1 and the 16 values of b
    const int n1 = n / kColN2;
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n1, (cuuint64_t)planes_in_buffer * kColN2};
    const cuuint64_t strides[2] = {(cuuint64_t)n * sizeof(float2), (cuuint64_t)n1 * n * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)kColW, 1, (cuuint32_t)kColN2};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, 3,
                              const_cast<float2*>(planes), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_colstack(const void* map, const StackArgs& a, int n1, int n2, float2* acc, const float* taper,
                            const double* sum_w, void* image, unsigned long long* err, cudaStream_t s, int nchan)
{
    if (a.nk <= 0 || nchan <= 0) return cudaSuccess;
    if (nchan > 1 && !a.chan_screen) return cudaErrorInvalidValue;
    if (nchan > 65535) return cudaErrorInvalidValue;
    if (n2 != kColN2 || (int64_t)n1 * n2 != a.n || a.n % kColW != 0) return cudaErrorInvalidValue;
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_colstack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    const dim3 grid((unsigned)(a.n / kColW), (unsigned)n1, (unsigned)nchan);
    k_colstack<<<grid, kColThreads, kColSmem, s>>>(*reinterpret_cast<const CUtensorMap*>(map), a, n1, acc, taper,
                                                   sum_w, image, err);
    return cudaGetLastError();
}

}  // namespace rick
