// rick_grid.cu -- convolutional gridding, Eq. 3 of the paper (sub-step 2 of
// step 2 in Sec. 2.1), and the taper used for grid correction.
//
// The counting sort of rick_prep.cu lists every (measurement, tile) pair whose
// S x S footprint touches a T x T tile of a w-plane, with the measurement's
// weighted, tap-normalised visibility.  Here each tile is owned by one warp
// (k_grid_tiles): the warp accumulates its entries into a private copy of the
// tile in shared memory and writes the whole tile once with coalesced 16-byte
// stores -- also when it is empty, so the planes need no memset and HBM sees
// each plane byte once.  No atomics, global or shared:
//   * lanes 0..15 evaluate the u taps and lanes 16..31 the v taps of one
//     entry (degree-10 polynomials, coefficients held in registers), then
//     every lane takes the (row, column) taps of its footprint cells by
//     shuffle, so one entry's S^2 cells are spread over the 32 lanes;
//   * a warp's cells for one entry are distinct, and the tile's row pitch P
//     is chosen with P = S (mod 16), which puts the 16 cells of each
//     half-warp in 16 different 8-byte bank pairs: read-modify-write of the
//     footprint is conflict-free;
//   * a __syncwarp between entries orders one entry's stores before the next
//     entry's loads.
// Tiles with more than kHeavyEntries entries (the dense centre of the uv
// plane) would serialise on one warp: k_grid_tiles writes them as zeros and
// lists them as chunks of at most kHeavyEntries entries, and k_grid_chunks
// gives every chunk to a warp, which adds its private tile into the plane
// with vector atomic adds.  Entries are loaded 32 at a time (one coalesced
// 512-byte load per warp) and broadcast by shuffle.  The fftshift
// checkerboard (-1)^(ju+jv) is folded into the tap signs.
#include "rick_internal.cuh"

namespace rick {
namespace {

constexpr int kHeavyEntries = 256;

int sm_count_grid()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// Row pitch (in cells) of a shared-memory tile: >= T and = S (mod 16).
__host__ __device__ __forceinline__ int tile_pitch(int T, int S) { return T + (((S - T) % 16) + 16) % 16; }

int light_warps(int T) { return T <= 16 ? 8 : (T <= 32 ? 4 : 1); }

// Per-lane constants: the footprint cells (slots) this lane updates for
// every entry: slot s is tap index lane + 32 s, at footprint row sr, column sc.
template <int S>
struct LaneSlots {
    static constexpr int kSlots = (S * S + 31) / 32;
    int sr[kSlots], sc[kSlots];
    bool ok[kSlots];

    __device__ __forceinline__ void init(int lane)
    {
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int i = lane + 32 * s;
            ok[s] = i < S * S;
            sr[s] = ok[s] ? i / S : 0;
            sc[s] = ok[s] ? i % S : 0;
        }
    }
};

// Per-warp staging of 32 entries in shared memory: their signed taps and a
// header (first cell relative to the tile origin, weighted visibility).
template <int S>
struct Stage {
    static constexpr int kStride = S <= 8 ? 8 : 16;
    float gu[32 * kStride];
    float gv[32 * kStride];
    float4 head[32];
};

// Shared memory of one warp: its tile (T rows of pitch P cells) and its stage.
template <int S>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int T)
{
    return (size_t)T * tile_pitch(T, S) * sizeof(float2) + sizeof(Stage<S>);
}

// Accumulate entries [b, e) of one sorted list into the warp's tile.  Rounds
// of 32 entries: (1) each lane takes one entry (coalesced 16-byte loads) and
// evaluates its 2S taps (degree-10 polynomials with uniform coefficients from
// the constant bank) with the checkerboard signs folded in, into the stage;
// (2) the warp walks the 32 entries, every lane updating its slots' cells.
// Within one entry the lanes' cells are distinct and, with pitch P = S
// (mod 16), in distinct bank pairs; a __syncwarp orders consecutive entries.
template <int S>
__device__ __forceinline__ void warp_grid_range(const GridCfg& c, const float4* __restrict__ ent, uint32_t b,
                                                uint32_t e, int u0, int v0, float2* tile, Stage<S>& st, int P,
                                                const LaneSlots<S>& ls, int lane, int shift)
{
    constexpr int K = Stage<S>::kStride;
    const unsigned T = (unsigned)c.T;
    for (uint32_t j0 = b; j0 < e; j0 += 32) {
        const uint32_t j = j0 + lane;
        if (j < e) {
            const float4 r = __ldg(ent + j);
            const int fu = first_cell(c, r.x), fv = first_cell(c, r.y);
            const float zu = __fmaf_rn(2.0f, __fsub_rn(__fsub_rn(r.x, c.half_s), (float)(fu - 1)), -1.0f);
            const float zv = __fmaf_rn(2.0f, __fsub_rn(__fsub_rn(r.y, c.half_s), (float)(fv - 1)), -1.0f);
#pragma unroll
            for (int t = 0; t < S; ++t) {
                float a = c.coef[t][kPolyTerms - 1], bb = c.coef[t][kPolyTerms - 1];
#pragma unroll
                for (int k = kPolyTerms - 2; k >= 0; --k) {
                    a = __fmaf_rn(a, zu, c.coef[t][k]);
                    bb = __fmaf_rn(bb, zv, c.coef[t][k]);
                }
                if (shift) {
                    if ((fu + t) & 1) a = -a;
                    if ((fv + t) & 1) bb = -bb;
                }
                st.gu[lane * K + t] = a;
                st.gv[lane * K + t] = bb;
            }
            st.head[lane] = make_float4(__int_as_float(fu - u0), __int_as_float(fv - v0), r.z, r.w);
        }
        __syncwarp();
        const int cnt = (e - j0 < 32u) ? (int)(e - j0) : 32;
        for (int q = 0; q < cnt; ++q) {
            const float4 h = st.head[q];
            const int lu = __float_as_int(h.x), lv = __float_as_int(h.y);
#pragma unroll
            for (int sl = 0; sl < LaneSlots<S>::kSlots; ++sl) {
                const unsigned row = (unsigned)(lv + ls.sr[sl]), col = (unsigned)(lu + ls.sc[sl]);
                if (ls.ok[sl] && row < T && col < T) {
                    const float wgt = st.gu[q * K + ls.sc[sl]] * st.gv[q * K + ls.sr[sl]];
                    float2* cell = tile + row * P + col;
                    float2 x = *cell;
                    x.x = __fmaf_rn(h.z, wgt, x.x);
                    x.y = __fmaf_rn(h.w, wgt, x.y);
                    *cell = x;
                }
            }
            __syncwarp();
        }
    }
}

struct TileGeom {
    int64_t tg;       // global tile id
    int kl;           // plane within the pass
    int u0, v0, wu, wv;
};

__device__ __forceinline__ TileGeom tile_geom(const GridCfg& c, int k0, int64_t tl)
{
    TileGeom g;
    g.kl = (int)(tl / c.ntp);
    const int rem = (int)(tl - (int64_t)g.kl * c.ntp);
    const int tv = rem / c.ntu, tu = rem - tv * c.ntu;
    g.tg = (int64_t)(k0 + g.kl) * c.ntp + rem;
    g.u0 = tu * c.T;
    g.v0 = tv * c.T;
    g.wu = min(c.T, c.n - g.u0);
    g.wv = min(c.T, c.n - g.v0);
    return g;
}

// Write (or zero) the valid part of a tile: 16 lanes per 256-byte row segment.
template <bool kZero>
__device__ __forceinline__ void store_tile(const GridCfg& c, const TileGeom& g, float2* P0, const float2* tile,
                                           int P, int tid, int nthreads)
{
    const int half = c.T >> 1;
    for (int i = tid; i < c.T * half; i += nthreads) {
        const int row = i / half, col = (i - row * half) * 2;
        if (row < g.wv && col < g.wu) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!kZero) {
                const float2 a = tile[row * P + col], b = tile[row * P + col + 1];
                v = make_float4(a.x, a.y, b.x, b.y);
            }
            *reinterpret_cast<float4*>(P0 + (int64_t)(g.v0 + row) * c.n + g.u0 + col) = v;
        }
    }
}

// Initialise a tile copy: zeros, or the plane's current values (accumulating pass).
__device__ __forceinline__ void init_tile(const GridCfg& c, const TileGeom& g, const float2* P0, float2* tile, int P,
                                          bool from_plane, int tid, int nthreads)
{
    if (!from_plane) {
        float4* t4 = reinterpret_cast<float4*>(tile);
        for (int i = tid; i < (c.T * P) / 2; i += nthreads) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    for (int i = tid; i < c.T * P; i += nthreads) {
        const int row = i / P, col = i - row * P;
        float2 x = make_float2(0.f, 0.f);
        if (row < g.wv && col < g.wu) x = P0[(int64_t)(g.v0 + row) * c.n + g.u0 + col];
        tile[i] = x;
    }
}

template <int S>
__global__ void __launch_bounds__(256) k_grid_tiles(GridCfg c, ChunkList ch, int k0, int64_t ntl, int shift,
                                                    int accumulate, float2* __restrict__ planes,
                                                    uint32_t* __restrict__ heavy, uint32_t heavy_cap)
{
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t tl = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (tl >= ntl) return;
    const int P = tile_pitch(c.T, S);
    unsigned char* mine = reinterpret_cast<unsigned char*>(smem4) + (size_t)wid * warp_smem_bytes<S>(c.T);
    float2* tile = reinterpret_cast<float2*>(mine);
    Stage<S>& st = *reinterpret_cast<Stage<S>*>(mine + (size_t)c.T * P * sizeof(float2));
    const TileGeom g = tile_geom(c, k0, tl);
    float2* P0 = planes + (int64_t)g.kl * c.n * c.n;

    uint32_t nent = 0;
    for (int q = 0; q < ch.count; ++q) nent += ch.off[q][g.tg + 1] - ch.off[q][g.tg];
    if (nent > (uint32_t)kHeavyEntries && ch.count == 1) {
        // many entries: hand the tile to k_grid_chunks as chunks of at most
        // kHeavyEntries entries, which add into the plane; the tile starts
        // at zero unless this pass accumulates onto earlier chunks
        const uint32_t nchunks = (nent + kHeavyEntries - 1) / kHeavyEntries;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(heavy, nchunks);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + nchunks <= heavy_cap) {
            for (uint32_t k = lane; k < nchunks; k += 32) {
                heavy[1 + 2 * (base + k)] = (uint32_t)tl;
                heavy[2 + 2 * (base + k)] = k;
            }
            if (!accumulate) store_tile<true>(c, g, P0, nullptr, P, lane, 32);
            return;
        }
        // no room in the chunk list: mark the reserved slots that do exist as
        // empty, and grid the tile here (correct, slower)
        for (uint32_t k = base + lane; k < heavy_cap; k += 32) heavy[1 + 2 * k] = 0xffffffffu;
    }
    if (nent == 0 && !accumulate) {
        store_tile<true>(c, g, P0, nullptr, P, lane, 32);
        return;
    }
    init_tile(c, g, P0, tile, P, accumulate != 0, lane, 32);
    __syncwarp();
    LaneSlots<S> ls;
    ls.init(lane);
    for (int q = 0; q < ch.count; ++q)
        warp_grid_range<S>(c, ch.ent[q], ch.off[q][g.tg], ch.off[q][g.tg + 1], g.u0, g.v0, tile, st, P, ls, lane,
                           shift);
    __syncwarp();
    store_tile<false>(c, g, P0, tile, P, lane, 32);
}

// Chunks of the tiles with many entries: one warp per chunk, private tile in
// shared memory, flushed into the plane with vector atomic adds (the tile's
// cells were zeroed by k_grid_tiles, which ran before on the same stream).
template <int S>
__global__ void __launch_bounds__(256) k_grid_chunks(GridCfg c, ChunkList ch, int k0, int shift,
                                                     float2* __restrict__ planes, const uint32_t* __restrict__ heavy,
                                                     uint32_t heavy_cap)
{
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int P = tile_pitch(c.T, S);
    unsigned char* mine = reinterpret_cast<unsigned char*>(smem4) + (size_t)wid * warp_smem_bytes<S>(c.T);
    float2* tile = reinterpret_cast<float2*>(mine);
    Stage<S>& st = *reinterpret_cast<Stage<S>*>(mine + (size_t)c.T * P * sizeof(float2));
    LaneSlots<S> ls;
    ls.init(lane);
    const uint32_t count = min(heavy[0], heavy_cap);
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t it = blockIdx.x * (blockDim.x >> 5) + wid; it < count; it += nwarps) {
        const uint32_t tl32 = heavy[1 + 2 * it];
        if (tl32 == 0xffffffffu) continue;  // slot of a tile gridded by k_grid_tiles itself
        const int64_t tl = tl32;
        const uint32_t k = heavy[2 + 2 * it];
        const TileGeom g = tile_geom(c, k0, tl);
        float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
        const uint32_t b0 = ch.off[0][g.tg], e0 = ch.off[0][g.tg + 1];
        const uint32_t b = b0 + k * kHeavyEntries;
        const uint32_t e = min(e0, b + kHeavyEntries);
        init_tile(c, g, P0, tile, P, false, lane, 32);
        __syncwarp();
        warp_grid_range<S>(c, ch.ent[0], b, e, g.u0, g.v0, tile, st, P, ls, lane, shift);
        __syncwarp();
        for (int i = lane; i < c.T * c.T; i += 32) {
            const int row = i / c.T, col = i - row * c.T;
            if (row < g.wv && col < g.wu) {
                const float2 x = tile[row * P + col];
                if (x.x != 0.f || x.y != 0.f) atomicAdd(P0 + (int64_t)(g.v0 + row) * c.n + g.u0 + col, x);
            }
        }
        __syncwarp();
    }
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int S>
cudaError_t launch_grid_s(const GridCfg& c, const ChunkList& ch, int k0, int nk, bool shift, bool accumulate,
                          float2* planes, uint32_t* heavy, cudaStream_t s)
{
    const int64_t ntl = (int64_t)nk * c.ntp;
    if (ntl <= 0) return cudaSuccess;
    const size_t tile_bytes = warp_smem_bytes<S>(c.T);
    const int wl = light_warps(c.T);
    const int64_t nblocks = (ntl + wl - 1) / wl;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    // heavy: [count, (tile, chunk) pairs]; it has 1 + ntl words
    const uint32_t cap = (uint32_t)(ntl / 2);
    cudaError_t e = cudaMemsetAsync(heavy, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if ((e = allow_smem(k_grid_tiles<S>, tile_bytes * wl)) != cudaSuccess) return e;
    if ((e = allow_smem(k_grid_chunks<S>, tile_bytes * wl)) != cudaSuccess) return e;
    k_grid_tiles<S><<<(unsigned)nblocks, 32 * wl, tile_bytes * wl, s>>>(c, ch, k0, ntl, shift ? 1 : 0,
                                                                       accumulate ? 1 : 0, planes, heavy, cap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_grid_chunks<S><<<(unsigned)(4 * sm_count_grid()), 32 * wl, tile_bytes * wl, s>>>(c, ch, k0, shift ? 1 : 0,
                                                                                        planes, heavy, cap);
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
                        bool accumulate, uint32_t* heavy, float2* planes, cudaStream_t s)
{
    switch (c.S) {
#define RICK_GRID_CASE(SS) \
    case SS: return launch_grid_s<SS>(c, ch, k0, nk, shift_sign, accumulate, planes, heavy, s);
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
