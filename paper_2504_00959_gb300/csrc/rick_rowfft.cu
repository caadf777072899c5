// rick_rowfft.cu -- the row transforms of the w-planes in one pass over the
// planes (step 3 of the workflow, Sec. 2.1: the 2D FFT of every plane; the
// columns are transformed by k_colfft and k_colstack).
//
// For n = 8192 and 16384 a row (64 or 128 KB of complex values) fits in the
// shared memory of one SM, so each row is read from HBM once and written
// once: k_rowfft is a persistent kernel, one block per SM, that brings a row
// in with one bulk copy (TMA, completing on an mbarrier), transforms it in
// shared memory and stores it from registers, issuing the next row's copy as
// soon as its last pass has read the buffer.
//
// The n-point DFT (n = 16 Q1, Q1 = 16 Q2, Q2 = 16 Q3 = 16 R, R = 4 or 2),
// with X[f], f = k1 + 16 (k2 + 16 (k3 + 16 k4)):
//   pass 1  thread a' < Q1: 16-point DFT over a1 of x[Q1 a1 + a'], times
//           w_n^(a' k1) -> block k1, offset a'
//   pass 2  thread (k1, a'' < Q2): 16-point DFT over a2 of block k1's
//           elements Q2 a2 + a'', times w_Q1^(a'' k2) -> offset Q2 k2 + a''
//   pass 3  thread (k1, k2, a''' < R): 16-point DFT over a3 of offsets
//           Q2 k2 + R a3 + a''', times w_Q2^(a''' k3) -> Q2 k2 + R k3 + a'''
//   pass 4  group (k1, k2, k3): R-point DFT over a''' -> X[f], stored.
// The bulk copy lands the row in natural order; from pass 1 on the blocks of
// Q1 elements are padded by one element (position p -> p + p / Q1), and the
// lanes of every half warp take 16 consecutive k1, so every shared-memory
// access of passes 2-4 hits 16 different 8-byte bank pairs, and every
// global store of a half warp is 16 consecutive values (128 bytes).  Each
// pass reads all its values, synchronises, then writes (the in-place
// positions of a pass are read by other threads).  Twiddles w_n^e come from
// two 128-entry tables in shared memory, w_n^e = lo[e mod 128] hi[e / 128].
#include "rick_internal.cuh"
#include "rick_tma.cuh"

#include <cmath>

namespace rick {
namespace {

constexpr unsigned long long kRfWaitNs = 1000000000ull;  // bound of one wait: 1 s

__device__ __forceinline__ float2 r_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 r_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 r_mul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <int SIGN>
__device__ __forceinline__ float2 r_rot(float2 a)  // times (s i)
{
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int SIGN>
__device__ __forceinline__ void r_dft4(float2& x0, float2& x1, float2& x2, float2& x3)
{
    const float2 a0 = r_add(x0, x2), a2 = r_sub(x0, x2);
    const float2 a1 = r_add(x1, x3), a3 = r_rot<SIGN>(r_sub(x1, x3));
    x0 = r_add(a0, a1);
    x2 = r_sub(a0, a1);
    x1 = r_add(a2, a3);
    x3 = r_sub(a2, a3);
}

__device__ __forceinline__ float2 r_w16(int k, int sign)
{
    const float c[10] = {1.0f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
                         -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128676f, -1.0f,
                         -0.92387953251128676f};
    const float s[10] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128676f, 1.0f,
                         0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
                         -0.38268343236508977f};
    return make_float2(c[k], sign * s[k]);
}

// 16-point DFT, natural order in and out (16 = 4 x 4, as in k_colfft)
template <int SIGN>
__device__ __forceinline__ void r_dft16(float2 (&v)[16])
{
    float2 t[4][4];
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2) {
        float2 a0 = v[c2], a1 = v[4 + c2], a2 = v[8 + c2], a3 = v[12 + c2];
        r_dft4<SIGN>(a0, a1, a2, a3);
        t[c2][0] = a0;
        t[c2][1] = c2 ? r_mul(a1, r_w16(c2, SIGN)) : a1;
        t[c2][2] = c2 ? r_mul(a2, r_w16(2 * c2, SIGN)) : a2;
        t[c2][3] = c2 ? r_mul(a3, r_w16(3 * c2, SIGN)) : a3;
    }
#pragma unroll
    for (int j1 = 0; j1 < 4; ++j1) {
        float2 a0 = t[0][j1], a1 = t[1][j1], a2 = t[2][j1], a3 = t[3][j1];
        r_dft4<SIGN>(a0, a1, a2, a3);
        v[j1] = a0;
        v[j1 + 4] = a1;
        v[j1 + 8] = a2;
        v[j1 + 12] = a3;
    }
}

// w_n^e for 0 <= e < n (n <= 16384): lo[e & 127] * hi[e >> 7], the tables
// hold exp(+2 pi i j / n) and exp(+2 pi i 128 j / n); conjugated for SIGN < 0
template <int SIGN>
__device__ __forceinline__ float2 r_twiddle(const float2* lo, const float2* hi, int e)
{
    float2 t = r_mul(lo[e & 127], hi[e >> 7]);
    if (SIGN < 0) t.y = -t.y;
    return t;
}

template <int N>
struct RowShape {
    static constexpr int Q1 = N / 16, Q2 = Q1 / 16, R = Q2 / 16;
    static constexpr int kThreads = Q1;
    static constexpr int kPadded = N + 16;                   // one pad element per block of Q1
    static constexpr size_t kSmem = (size_t)kPadded * 8 + 2 * 128 * 8 + 16;
};

__device__ __forceinline__ int pad_q(int p, int log2q1) { return p + (p >> log2q1); }

// grid: one block per SM (persistent), RowShape<N>::kThreads threads; rows
// r = blockIdx.x, blockIdx.x + gridDim.x, ... of the nrows rows at `rows`.
// tw: [256] = lo[128] then hi[128] (exp(+2 pi i j / N), exp(+2 pi i 128 j / N)).
// err: bit 2 set when a bounded wait ran out.
template <int N, int SIGN>
__global__ void __launch_bounds__(RowShape<N>::kThreads, 1)
    k_rowfft(float2* __restrict__ rows, int64_t nrows, const float2* __restrict__ tw, unsigned long long wait_ns,
             unsigned long long* __restrict__ err)
{
    using S = RowShape<N>;
    constexpr int Q1 = S::Q1, Q2 = S::Q2, R = S::R;
    constexpr int L1 = (Q1 == 1024) ? 10 : 9;  // log2 Q1
    static_assert((1 << L1) == Q1, "Q1 is 512 or 1024");
    extern __shared__ __align__(128) unsigned char rf_smem[];
    float2* buf = reinterpret_cast<float2*>(rf_smem);        // [S::kPadded]
    float2* lo = buf + S::kPadded;                             // [128]
    float2* hi = lo + 128;                                     // [128]
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(hi + 128);
    __shared__ int s_abort;

    const int t = threadIdx.x;
    const unsigned long long limit = wait_ns ? wait_ns : kRfWaitNs;
    for (int j = t; j < 256; j += S::kThreads) lo[j] = __ldg(tw + j);
    if (t == 0) {
        s_abort = 0;
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t r = blockIdx.x;
    if (r >= nrows) return;
    if (t == 0) {
        mbar_expect(smem_u32(bar), (uint32_t)(N * sizeof(float2)));
        bulk_load(smem_u32(buf), rows + r * N, (uint32_t)(N * sizeof(float2)), smem_u32(bar));
    }
    // thread roles (k1 on the 16 lanes of a half warp)
    const int k1 = t & 15, u = t >> 4;  // pass 2: a'' = u (< Q2); pass 3: k2 = u % 16, a''' = u / 16 (< R)
    uint32_t phase = 0;
    for (; r < nrows; r += gridDim.x) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), phase, &s_abort, limit));
        if (!ok) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        phase ^= 1;
        float2 v[16];
        // pass 1: thread a' = t
#pragma unroll
        for (int a1 = 0; a1 < 16; ++a1) v[a1] = buf[Q1 * a1 + t];
        __syncthreads();
        r_dft16<SIGN>(v);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            buf[pad_q(Q1 * k + t, L1)] = k ? r_mul(v[k], r_twiddle<SIGN>(lo, hi, t * k)) : v[k];
        __syncthreads();
        // pass 2: thread (k1, a'' = u), u < Q2
        {
            const int base = pad_q(Q1 * k1, L1) + u;
#pragma unroll
            for (int a2 = 0; a2 < 16; ++a2) v[a2] = buf[base + Q2 * a2];
            __syncthreads();
            r_dft16<SIGN>(v);
#pragma unroll
            for (int k = 0; k < 16; ++k)  // w_Q1^(a'' k2) = w_n^(16 a'' k2)
                buf[base + Q2 * k] = k && u ? r_mul(v[k], r_twiddle<SIGN>(lo, hi, 16 * u * k)) : v[k];
            __syncthreads();
        }
        // pass 3: thread (k1, k2 = u % 16, a''' = u / 16), a''' < R
        {
            const int k2 = u & 15, a3p = u >> 4;
            const int base = pad_q(Q1 * k1, L1) + Q2 * k2 + a3p;
#pragma unroll
            for (int a3 = 0; a3 < 16; ++a3) v[a3] = buf[base + R * a3];
            __syncthreads();
            r_dft16<SIGN>(v);
#pragma unroll
            for (int k = 0; k < 16; ++k)  // w_Q2^(a''' k3) = w_n^(256 a''' k3)
                buf[base + R * k] = k && a3p ? r_mul(v[k], r_twiddle<SIGN>(lo, hi, 256 * a3p * k)) : v[k];
            __syncthreads();
        }
        // pass 4: groups (k1, k2, k3), 4096 of them, R values each
        constexpr int kGroups = 4096 / S::kThreads;
        float2 g[kGroups][R];
#pragma unroll
        for (int q = 0; q < kGroups; ++q) {
            const int gi = u + (S::kThreads / 16) * q;  // (k2, k3) = (gi % 16, gi / 16)
            const int base = pad_q(Q1 * k1, L1) + Q2 * (gi & 15) + R * (gi >> 4);
#pragma unroll
            for (int j = 0; j < R; ++j) g[q][j] = buf[base + j];
        }
        __syncthreads();
        // the buffer is free: bring in the next row while this one finishes
        if (t == 0 && r + gridDim.x < nrows) {
            mbar_expect(smem_u32(bar), (uint32_t)(N * sizeof(float2)));
            bulk_load(smem_u32(buf), rows + (r + gridDim.x) * N, (uint32_t)(N * sizeof(float2)), smem_u32(bar));
        }
        float2* out = rows + r * N;
#pragma unroll
        for (int q = 0; q < kGroups; ++q) {
            const int gi = u + (S::kThreads / 16) * q;
            if constexpr (R == 4) {
                r_dft4<SIGN>(g[q][0], g[q][1], g[q][2], g[q][3]);
            } else {
                const float2 a = g[q][0];
                g[q][0] = r_add(a, g[q][1]);
                g[q][1] = r_sub(a, g[q][1]);
            }
#pragma unroll
            for (int k4 = 0; k4 < R; ++k4) out[k1 + 16 * gi + 4096 * k4] = g[q][k4];
        }
    }
    if (s_abort) {
        if (t == 0) {
            atomicOr(err, 4ull);
            // the copy this block issued last: let it land before leaving
            const unsigned long long t0 = global_ns();
            while (!mbar_try(smem_u32(bar), phase) && global_ns() - t0 <= limit) {
            }
        }
        __syncthreads();
    }
}

template <int N, int SIGN>
cudaError_t launch_rf(float2* planes, int nk, const float2* tw, unsigned long long wait_ns, unsigned long long* err,
                      cudaStream_t s)
{
    using S = RowShape<N>;
    static bool attr_done[64] = {false};
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done[dev]) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_rowfft<N, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
        if (e != cudaSuccess) return e;
        cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        attr_done[dev] = true;
    }
    const int64_t nrows = (int64_t)nk * N;
    const unsigned blocks = (unsigned)(nrows < sms[dev] ? nrows : sms[dev]);
    k_rowfft<N, SIGN><<<blocks, S::kThreads, S::kSmem, s>>>(planes, nrows, tw, wait_ns, err);
    return cudaGetLastError();
}

}  // namespace

bool rowfft_supported(int n) { return n == 8192 || n == 16384; }

void rowfft_tables(int n, float2* tw256)
{
    for (int j = 0; j < 128; ++j) {
        const double a = 6.283185307179586476925 * (double)j / (double)n;
        const double b = 6.283185307179586476925 * (double)(128 * j) / (double)n;
        tw256[j] = make_float2((float)std::cos(a), (float)std::sin(a));
        tw256[128 + j] = make_float2((float)std::cos(b), (float)std::sin(b));
    }
}

cudaError_t launch_rowfft(float2* planes, int n, int nk, int sign, const float2* tw, unsigned long long wait_ns,
                          unsigned long long* err, cudaStream_t s)
{
    if (nk <= 0) return cudaSuccess;
    if (n == 16384) return sign > 0 ? launch_rf<16384, 1>(planes, nk, tw, wait_ns, err, s)
                                    : launch_rf<16384, -1>(planes, nk, tw, wait_ns, err, s);
    if (n == 8192) return sign > 0 ? launch_rf<8192, 1>(planes, nk, tw, wait_ns, err, s)
                                   : launch_rf<8192, -1>(planes, nk, tw, wait_ns, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace rick
