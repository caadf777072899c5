// rick_colfft.cu -- the first factor of the split column transform (step 3
// of the workflow, Sec. 2.1: the 2D FFT of every w-plane), one launch per
// plane group.
//
// With n = N1 * 16, row v = 16 a + b and output row y = f1 + N1 f2, the
// column transform of a plane (after its rows) is
//     X[f1 + N1 f2] = sum_b w_16^(b f2) (w_n^(b f1) Y[16 f1 + b]),
//     Y[16 f1 + b]  = sum_a x[16 a + b] w_N1^(a f1),
// (w_M = exp(s 2 pi i / M), s = +1 for imaging, -1 for the adjoint).  The
// planes of the split transform keep their rows in b-major order: grid row
// 16 a + b is memory row b N1 + a, so the N1 rows of one b are a contiguous
// run (a plane is [16][N1][n]).  This kernel computes Y in place: for each
// plane, each b and each strip of W adjacent columns, rows a = 0 .. N1-1 of
// that run are one 3D TMA box per 256 rows (the buffer viewed as
// [16 G][N1][n]) brought into shared memory ([a][W] complex values, 64- or
// 128-byte row segments), transformed there and written back to memory row
// b N1 + f1 (grid row 16 f1 + b).  With natural row order the rows of one
// column transform lie 16 rows apart across the whole plane, and a 16384^2
// plane's column pass reached ~0.73 of the copy bandwidth even without the
// arithmetic (1.01 in b-major order).  The last factor (over b) is fused
// with the w-screen and the plane sum in k_colstack, or applied to the
// planes by k_spreadcol in the adjoint.
//
// The N1-point transform (N1 = 16 .. 1024; 4 and 8 in one pass) runs in
// shared memory as
// N1 = 16 x Q:
//   pass A  for each a2 < Q: 16-point DFT over a1 (rows Q a1 + a2), times
//           w_N1^(a2 k1), written back in place (row Q k1 + a2);
//   pass B  for each k1: the Q-point DFT over a2 of rows Q k1 + a2, output
//           f1 = k1 + 16 kq -- directly (Q <= 16), or for Q = 16 r (N1 =
//           512, 1024) as a 16-point pass over c1 (a2 = r c1 + c2) times
//           w_Q^(c2 j1), stored transposed (row Q k1 + 16 c2 + j1) by the
//           warp that owns block k1, then an r-point pass over c2, output
//           kq = j1 + 16 j2.
// Every shared-memory access of a half warp covers 128 contiguous bytes or
// two adjacent 64-byte rows (no bank conflicts); the results go to global
// memory from registers (W columns of a row per group of W lanes).
#include "rick_internal.cuh"
#include "rick_tma.cuh"

#include <cudaTypedefs.h>

namespace rick {
namespace {

constexpr int kCfThreads = 256;
constexpr unsigned long long kCfWaitNs = 1000000000ull;  // bound of the load wait: 1 s
constexpr int kCfBoxRows = 256;                          // TMA box: at most 256 rows per copy

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// times (s i)
template <int SIGN>
__device__ __forceinline__ float2 c_rot(float2 a)
{
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-place DFTs of 2, 4, 8 and 16 points with exponent sign SIGN, natural
// order in and out.
template <int SIGN>
__device__ __forceinline__ void dft2(float2& a, float2& b)
{
    const float2 t = a;
    a = c_add(t, b);
    b = c_sub(t, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3)
{
    const float2 a0 = c_add(x0, x2), a2 = c_sub(x0, x2);
    const float2 a1 = c_add(x1, x3), a3 = c_rot<SIGN>(c_sub(x1, x3));
    x0 = c_add(a0, a1);
    x2 = c_sub(a0, a1);
    x1 = c_add(a2, a3);
    x3 = c_sub(a2, a3);
}

// w_8^k, k = 1, 3 (w_8^2 = s i)
constexpr float kR2 = 0.70710678118654752f;

template <int SIGN>
__device__ __forceinline__ void dft8(float2 (&v)[8])
{
    // 8 = 2 x 4: index 4 c1 + c2 -> output j1 + 2 j2 ... written as two
    // 4-point transforms over the even and odd samples and one radix-2 pass
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    // twiddles w_8^k on the odd transform
    const float s = (float)SIGN;
    o1 = c_mul(o1, make_float2(kR2, s * kR2));
    o2 = c_rot<SIGN>(o2);
    o3 = c_mul(o3, make_float2(-kR2, s * kR2));
    v[0] = c_add(e0, o0);
    v[4] = c_sub(e0, o0);
    v[1] = c_add(e1, o1);
    v[5] = c_sub(e1, o1);
    v[2] = c_add(e2, o2);
    v[6] = c_sub(e2, o2);
    v[3] = c_add(e3, o3);
    v[7] = c_sub(e3, o3);
}

// cos and sin of 2 pi k / 16, k = 0 .. 9
__device__ __forceinline__ float2 w16(int k, int sign)
{
    const float c[10] = {1.0f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
                         -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128676f, -1.0f,
                         -0.92387953251128676f};
    const float s[10] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128676f, 1.0f,
                         0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
                         -0.38268343236508977f};
    return make_float2(c[k], sign * s[k]);
}

template <int SIGN>
__device__ __forceinline__ void dft16(float2 (&v)[16])
{
    // 16 = 4 x 4: sample 4 c1 + c2; first 4-point DFTs over c1 (for each
    // c2), times w_16^(c2 j1), then over c2 (for each j1): output j1 + 4 j2
    float2 t[4][4];
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2) {
        float2 a0 = v[c2], a1 = v[4 + c2], a2 = v[8 + c2], a3 = v[12 + c2];
        dft4<SIGN>(a0, a1, a2, a3);
        t[c2][0] = a0;
        t[c2][1] = c2 ? c_mul(a1, w16(c2, SIGN)) : a1;
        t[c2][2] = c2 ? c_mul(a2, w16(2 * c2, SIGN)) : a2;
        t[c2][3] = c2 ? c_mul(a3, w16(3 * c2, SIGN)) : a3;
    }
#pragma unroll
    for (int j1 = 0; j1 < 4; ++j1) {
        float2 a0 = t[0][j1], a1 = t[1][j1], a2 = t[2][j1], a3 = t[3][j1];
        dft4<SIGN>(a0, a1, a2, a3);
        v[j1] = a0;
        v[j1 + 4] = a1;
        v[j1 + 8] = a2;
        v[j1 + 12] = a3;
    }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_small(float2 (&v)[R])
{
    if constexpr (R == 2) {
        dft2<SIGN>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft8<SIGN>(v);
    } else if constexpr (R == 16) {
        dft16<SIGN>(v);
    }
}

// twiddle w_N1^e with the kernel's sign from the block's shared copy of the
// table of exp(+2 pi i j / N1)
template <int SIGN>
__device__ __forceinline__ float2 twid(const float2* tw, int e)
{
    float2 t = tw[e];
    if (SIGN < 0) t.y = -t.y;
    return t;
}

// The N1 = 16 Q-point transform (N1 >= 16) of the block in shared memory
// ([N1][W] complex values), output f1 written to row f1 of the run at P.
template <int N1, int W, int SIGN>
__device__ __forceinline__ void colfft_two_pass(float2* __restrict__ buf, const float2* tw,
                                                float2* __restrict__ P, int n, int t)
{
    constexpr int Q = N1 / 16;
    // pass A: 16-point DFTs over a1 (rows Q a1 + a2), twiddle w_N1^(a2 k1)
    for (int it = t; it < Q * W; it += kCfThreads) {
        const int x = it % W, a2 = it / W;
        float2 v[16];
#pragma unroll
        for (int a1 = 0; a1 < 16; ++a1) v[a1] = buf[(Q * a1 + a2) * W + x];
        dft16<SIGN>(v);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            const float2 r = (k1 && a2) ? c_mul(v[k1], twid<SIGN>(tw, a2 * k1)) : v[k1];
            buf[(Q * k1 + a2) * W + x] = r;
        }
    }
    __syncthreads();

    if constexpr (Q <= 16) {
        // pass B: Q-point DFT over a2 (rows Q k1 + a2); output f1 = k1 + 16 kq
        for (int it = t; it < 16 * W; it += kCfThreads) {
            const int x = it % W, k1 = it / W;
            if constexpr (Q == 1) {
                P[(size_t)k1 * n + x] = buf[k1 * W + x];
            } else {
                float2 v[Q];
#pragma unroll
                for (int a2 = 0; a2 < Q; ++a2) v[a2] = buf[(Q * k1 + a2) * W + x];
                dft_small<Q, SIGN>(v);
#pragma unroll
                for (int kq = 0; kq < Q; ++kq) P[(size_t)(k1 + 16 * kq) * n + x] = v[kq];
            }
        }
    } else {
        // Q = 16 r.  Pass B1: the warp owning block k1 (Q rows) runs 16-point
        // DFTs over c1 (rows Q k1 + r c1 + c2), times w_Q^(c2 j1), and stores
        // them transposed, row Q k1 + 16 c2 + (j1 ^ c2): the XOR puts the
        // values of one j1 in different (row mod r) slots, so the half warps
        // of this pass (W columns x 2 values of c2) and of pass B2 (W columns
        // x 2 consecutive j1) each touch two adjacent rows' worth of banks
        constexpr int r = Q / 16;
        static_assert(r * W * 16 == 16 * 32 || r * W * 16 == 16 * 16, "one warp (or half) per block of Q rows");
        constexpr int kLanesPerBlock = r * W;  // 32 or 16
        const int lane = t & 31, wid = t >> 5;
        const int sub = lane / kLanesPerBlock, l = lane % kLanesPerBlock;
        const int x = l % W, c2 = l / W;
        constexpr int kBlocksPerWarp = 32 / kLanesPerBlock;
        for (int k1 = wid * kBlocksPerWarp + sub; k1 < 16; k1 += (kCfThreads / 32) * kBlocksPerWarp) {
            float2 v[16];
#pragma unroll
            for (int c1 = 0; c1 < 16; ++c1) v[c1] = buf[(Q * k1 + r * c1 + c2) * W + x];
            dft16<SIGN>(v);
            __syncwarp();
#pragma unroll
            for (int j1 = 0; j1 < 16; ++j1) {
                // w_Q^(c2 j1) = w_N1^(16 c2 j1)
                const float2 rr = (c2 && j1) ? c_mul(v[j1], twid<SIGN>(tw, 16 * c2 * j1)) : v[j1];
                buf[(Q * k1 + 16 * c2 + (j1 ^ c2)) * W + x] = rr;
            }
            __syncwarp();
        }
        __syncthreads();
        // pass B2: r-point DFTs over c2 (rows Q k1 + 16 c2 + (j1 ^ c2)); output
        // kq = j1 + 16 j2, f1 = k1 + 16 kq
        for (int it = t; it < 16 * 16 * W; it += kCfThreads) {
            const int xx = it % W, j1 = (it / W) % 16, k1 = it / (16 * W);
            float2 v[r];
#pragma unroll
            for (int q = 0; q < r; ++q) v[q] = buf[(Q * k1 + 16 * q + (j1 ^ q)) * W + xx];
            dft_small<r, SIGN>(v);
#pragma unroll
            for (int j2 = 0; j2 < r; ++j2)
                P[(size_t)(k1 + 16 * (j1 + 16 * j2)) * n + xx] = v[j2];
        }
    }
}

// grid (n / W, 16, planes of the group); block kCfThreads; dynamic shared
// memory N1 * W complex values, the N1 twiddles and one mbarrier.  tw:
// exp(+2 pi i j / N1), j < N1 (device; copied in with the block's data).
// err: bit 1 set when the load wait ran out.
template <int N1, int W, int SIGN>
__global__ void __launch_bounds__(kCfThreads) k_colfft(const __grid_constant__ CUtensorMap map,
                                                       const float2* __restrict__ tw, float2* __restrict__ planes,
                                                       int n, unsigned long long wait_ns,
                                                       unsigned long long* __restrict__ err)
{
    constexpr int kBox = N1 < kCfBoxRows ? N1 : kCfBoxRows;
    extern __shared__ __align__(128) unsigned char cf_smem[];
    float2* buf = reinterpret_cast<float2*>(cf_smem);  // [N1][W]
    float2* tws = buf + (size_t)N1 * W;                 // [N1] twiddles
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(tws + N1);
    __shared__ int s_abort;

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W, b = blockIdx.y, plane = blockIdx.z;
    const unsigned long long limit = wait_ns ? wait_ns : kCfWaitNs;
    if (t == 0) {
        s_abort = 0;
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        mbar_expect(smem_u32(bar), (uint32_t)((N1 * W + N1) * sizeof(float2)));
#pragma unroll
        for (int a0 = 0; a0 < N1; a0 += kBox)
            tma_load_3d(smem_u32(buf + (size_t)a0 * W), &map, x0, a0, plane * 16 + b, smem_u32(bar));
        bulk_load(smem_u32(tws), tw, (uint32_t)(N1 * sizeof(float2)), smem_u32(bar));
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), 0, &s_abort, limit));
    if (!ok) s_abort = 1;
    __syncthreads();
    if (s_abort) {
        // leave no bulk copy in flight into this block's shared memory
        if (t == 0) {
            atomicOr(err, 2ull);
            const unsigned long long t0 = global_ns();
            while (!mbar_try(smem_u32(bar), 0) && global_ns() - t0 <= limit) {
            }
        }
        __syncthreads();
        return;
    }

    // the run of rows b N1 .. b N1 + N1 - 1 of the plane, from column x0
    float2* P = planes + (size_t)plane * n * n + (size_t)b * N1 * n + x0;
    if constexpr (N1 < 16) {
        // a single N1-point DFT per column (n = 64, 128)
        for (int it = t; it < W; it += kCfThreads) {
            float2 v[N1];
#pragma unroll
            for (int a = 0; a < N1; ++a) v[a] = buf[a * W + it];
            dft_small<N1, SIGN>(v);
#pragma unroll
            for (int f1 = 0; f1 < N1; ++f1) P[(size_t)f1 * n + it] = v[f1];
        }
    } else {
        colfft_two_pass<N1, W, SIGN>(buf, tws, P, n, t);
    }
}

template <int N1, int W, int SIGN>
cudaError_t launch_cf(const void* map, const float2* tw, float2* planes, int n, int nk, unsigned long long wait_ns,
                      unsigned long long* err, cudaStream_t s)
{
    const size_t smem = (size_t)(N1 * W + N1) * sizeof(float2) + 16;
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_colfft<N1, W, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    const dim3 grid((unsigned)(n / W), 16u, (unsigned)nk);
    k_colfft<N1, W, SIGN><<<grid, kCfThreads, smem, s>>>(*reinterpret_cast<const CUtensorMap*>(map), tw, planes,
                                                          n, wait_ns, err);
    return cudaGetLastError();
}

// columns per block: 128-byte row segments up to N1 = 256 (32 KB), 64-byte
// ones for the longer transforms (64 KB at N1 = 1024, three blocks per SM)
template <int N1>
constexpr int cf_width()
{
    return N1 <= 256 ? 16 : 8;
}

}  // namespace

int colfft_width(int n1)
{
    return n1 <= 256 ? 16 : 8;
}

cudaError_t encode_colfft_map(void* map, const float2* planes, int n, int planes_in_buffer)
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
    const int n1 = n / 16;
    const int w = colfft_width(n1);
    // the plane buffer as [planes * 16][N1][n] 8-byte complex values: grid
    // row 16 a + b of plane p (memory row b N1 + a) is (a, 16 p + b)
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n1, (cuuint64_t)planes_in_buffer * 16};
    const cuuint64_t strides[2] = {(cuuint64_t)n * sizeof(float2), (cuuint64_t)n1 * n * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)(n1 < kCfBoxRows ? n1 : kCfBoxRows), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, 3,
                              const_cast<float2*>(planes), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_colfft(const void* map, const float2* tw, float2* planes, int n, int nk, int sign,
                          unsigned long long wait_ns, unsigned long long* err, cudaStream_t s)
{
    if (nk <= 0) return cudaSuccess;
    if (nk > 65535) return cudaErrorInvalidValue;
    const int n1 = n / 16;
#define RICK_CF_CASE(N1)                                                                                   \
    case N1:                                                                                               \
        return sign > 0 ? launch_cf<N1, cf_width<N1>(), 1>(map, tw, planes, n, nk, wait_ns, err, s)        \
                        : launch_cf<N1, cf_width<N1>(), -1>(map, tw, planes, n, nk, wait_ns, err, s);
    if (n != 16 * n1) return cudaErrorInvalidValue;
    switch (n1) {
        RICK_CF_CASE(4)
        RICK_CF_CASE(8)
        RICK_CF_CASE(16)
        RICK_CF_CASE(32)
        RICK_CF_CASE(64)
        RICK_CF_CASE(128)
        RICK_CF_CASE(256)
        RICK_CF_CASE(512)
        RICK_CF_CASE(1024)
        default: return cudaErrorInvalidValue;
    }
#undef RICK_CF_CASE
}

}  // namespace rick
