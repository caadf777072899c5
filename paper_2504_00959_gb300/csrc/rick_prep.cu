// rick_prep.cu -- sub-step 1 of gridding (Sec. 2.1: the measurements are
// gathered into one array per sector of the uv plane), done as a device
// counting sort by (w-plane, uv tile):
//   k_density  nearest-cell counts for uniform weighting
//   k_count    entries per tile (a footprint straddling tiles is listed in
//              every tile it touches)
//   k_scan_*   exclusive prefix sum of the counts -> tile start offsets
//   k_scatter  one 16-byte entry (pu, pv, s*Re V, s*Im V), s = weight / (sum of
//              u taps * sum of v taps), per (measurement, tile), written at
//              its tile's cursor; weight sum and counters.
// Grids are sized to the SM count; each block takes a contiguous range of the
// measurements (split at channel boundaries in batched imaging) and reads it
// coalesced; writes of entries are scattered 16-byte stores.
#include "rick_internal.cuh"

namespace rick {
namespace {

int sm_count()
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

constexpr int kPrepThreads = 256;

int prep_blocks(int64_t m, int bpsm = 8)
{
    int64_t want = (m + kPrepThreads - 1) / kPrepThreads;
    int64_t cap = (int64_t)sm_count() * (bpsm > 0 ? bpsm : 8);
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

struct Inputs {
    const float* u;
    const float* v;
    const float* w;
    const float* wt;
    const float2* vis;
};

__device__ __forceinline__ bool load_and_place(const GridCfg& c, const Inputs& in, int64_t i, int chan, Place& p,
                                               float& wi, float2& V)
{
    wi = in.wt ? __ldg(in.wt + i) : 1.0f;
    V = __ldg(in.vis + i);
    if (!place(c, __ldg(in.u + i), __ldg(in.v + i), __ldg(in.w + i), p, chan)) return false;
    if (p.conj) V.y = -V.y;
    return finite_value(wi, V);
}

// Each block takes one contiguous range of the m measurements and walks it
// channel by channel (one segment when there is a single channel): body(chan,
// i0, i1) is called for every non-empty segment, by all threads of the block.
template <typename Body>
__device__ __forceinline__ void for_each_segment(const GridCfg& c, int64_t m, Body&& body)
{
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    int64_t r0 = (int64_t)blockIdx.x * per;
    const int64_t r1 = r0 + per < m ? r0 + per : m;
    if (r0 >= r1) return;
    int chan = 0;
    if (c.nchan > 1) {
        int lo = 0, hi = c.nchan - 1;  // last channel whose first measurement is <= r0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(c.chan_off + mid) <= r0) lo = mid; else hi = mid - 1;
        }
        chan = lo;
    }
    while (r0 < r1) {
        const int64_t end = (c.nchan > 1) ? min(r1, (int64_t)__ldg(c.chan_off + chan + 1)) : r1;
        if (end > r0) body(chan, r0, end);
        r0 = end > r0 ? end : r0;
        ++chan;
        if (chan >= c.nchan && r0 < r1) break;  // measurements past the last channel: none by construction
    }
}

__global__ void __launch_bounds__(kPrepThreads) k_density(GridCfg c, Inputs in, int64_t m,
                                                          uint32_t* __restrict__ density)
{
    for_each_segment(c, m, [&](int chan, int64_t i0, int64_t i1) {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            Place p;
            float wi;
            float2 V;
            if (!load_and_place(c, in, i, chan, p, wi, V)) continue;
            atomicAdd(density + (int64_t)nearest_cell(c, p.pv) * c.n + nearest_cell(c, p.pu), 1u);
        }
    });
}

// Tiles of plane `plane` touched by the uv footprint of a placed measurement: t[0] always, t[1]
// (right neighbour), t[2] (lower), t[3] (lower right) when the footprint
// straddles; -1 otherwise.
__device__ __forceinline__ void footprint_tiles(const GridCfg& c, const Place& p, int plane, int64_t (&t)[4])
{
    const int tu0 = p.fu >> c.log2T, tu1 = (p.fu + c.S - 1) >> c.log2T;
    const int tv0 = p.fv >> c.log2T, tv1 = (p.fv + c.S - 1) >> c.log2T;
    const int64_t base = (int64_t)plane * c.ntp;
    t[0] = base + tv0 * c.ntu + tu0;
    t[1] = tu1 != tu0 ? base + tv0 * c.ntu + tu1 : -1;
    t[2] = tv1 != tv0 ? base + tv1 * c.ntu + tu0 : -1;
    t[3] = (tu1 != tu0 && tv1 != tv0) ? base + tv1 * c.ntu + tu1 : -1;
}

// Measurements per thread and loop trip: their loads, and then their atomics,
// are in flight together.  Two rather than four: the scatter then needs 78
// instead of 128 registers and runs three CTAs per SM instead of two
// (measured 0.426 -> 0.392 ms at 4096^2 x 32 x 1e7, 34.1 -> 33.2 ms at
// 16384^2 x 128 x 2e8).
constexpr int kVisPerThread = 2;

__global__ void __launch_bounds__(kPrepThreads) k_count(GridCfg c, Inputs in, int64_t m,
                                                        uint32_t* __restrict__ counts)
{
    for_each_segment(c, m, [&](int chan, int64_t i0, int64_t i1) {
        for (int64_t ib = i0 + threadIdx.x; ib < i1; ib += (int64_t)kVisPerThread * blockDim.x) {
            Place p[kVisPerThread];
            bool ok[kVisPerThread];
#pragma unroll
            for (int q = 0; q < kVisPerThread; ++q) {
                const int64_t i = ib + (int64_t)q * blockDim.x;
                float wi;
                float2 V;
                ok[q] = i < i1 && load_and_place(c, in, i, chan, p[q], wi, V);
            }
#pragma unroll
            for (int q = 0; q < kVisPerThread; ++q) {
                if (!ok[q]) continue;
                // the measurement's planes: its own (Sw = 1) or its w-footprint
                for (int tw = 0; tw < c.Sw; ++tw) {
                    const int plane = p[q].k + tw;
                    if (plane < c.plane_lo || plane >= c.plane_hi) continue;
                    int64_t t[4];
                    footprint_tiles(c, p[q], plane, t);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (t[r] >= 0) atomicAdd(counts + t[r] * c.cstride, 1u);
                }
            }
        }
    });
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum of one float over the block (all threads call it); result valid in thread 0.
__device__ __forceinline__ float block_sum(float x)
{
    __shared__ float s[kPrepThreads / 32];
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s[wid] = x;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int j = 0; j < kPrepThreads / 32; ++j) t += s[j];
    return t;
}

// chan_sw[chan] accumulates the weight sum of each channel (one entry when
// there is a single channel).
__global__ void __launch_bounds__(kPrepThreads) k_scatter(GridCfg c, Inputs in, int64_t m,
                                                          const uint32_t* __restrict__ density,
                                                          uint32_t* __restrict__ cursor,
                                                          float4* __restrict__ entries, Counters* ctr,
                                                          double* __restrict__ chan_sw)
{
    unsigned gridded = 0, dropped = 0, nent = 0;
    for_each_segment(c, m, [&](int chan, int64_t i0, int64_t i1) {
        float sw = 0.0f;
        for (int64_t ib = i0 + threadIdx.x; ib < i1; ib += (int64_t)kVisPerThread * blockDim.x) {
            Place p[kVisPerThread];
            float wi[kVisPerThread];
            float2 V[kVisPerThread];
            bool ok[kVisPerThread];
#pragma unroll
            for (int q = 0; q < kVisPerThread; ++q) {
                const int64_t i = ib + (int64_t)q * blockDim.x;
                ok[q] = false;
                if (i < i1) {
                    ok[q] = load_and_place(c, in, i, chan, p[q], wi[q], V[q]);
                    if (!ok[q]) ++dropped;
                }
            }
            // the gridder reads the visibility already weighted and divided by
            // the two tap sums (normalised taps), once per measurement here
            // instead of once per (measurement, tile) entry there
            float4 rec[kVisPerThread];
            uint32_t slot[kVisPerThread][4];
            int64_t t[kVisPerThread][4];
#pragma unroll
            for (int q = 0; q < kVisPerThread; ++q) {
                if (!ok[q]) continue;
                if (c.uniform) {
                    const uint32_t cnt =
                        __ldg(density + (int64_t)nearest_cell(c, p[q].pv) * c.n + nearest_cell(c, p[q].pu));
                    wi[q] = wi[q] / (float)cnt;
                }
                const float scale = wi[q] / (tap_sum(c, p[q].pu, p[q].fu) * tap_sum(c, p[q].pv, p[q].fv));
                rec[q] = make_float4(p[q].pu, p[q].pv, scale * V[q].x, scale * V[q].y);
                sw += wi[q];
                ++gridded;
                if (c.Sw > 1) {
                    // w-footprint: one set of entries per plane, the w-tap in the scale
                    const float hn = w_tap_norm(c, p[q]);
                    for (int tw = 0; tw < c.Sw; ++tw) {
                        const int plane = p[q].k + tw;
                        if (plane < c.plane_lo || plane >= c.plane_hi) continue;
                        const float ht = w_kernel(c, __fsub_rn((float)plane, p[q].pw)) * hn;
                        const float4 rw = make_float4(rec[q].x, rec[q].y, ht * rec[q].z, ht * rec[q].w);
                        int64_t tt[4];
                        footprint_tiles(c, p[q], plane, tt);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            if (tt[r] >= 0) {
                                entries[atomicAdd(cursor + tt[r] * c.cstride, 1u)] = rw;
                                ++nent;
                            }
                    }
                    ok[q] = false;  // written: skip the nearest-plane stores below
                    continue;
                }
                if (p[q].k < c.plane_lo || p[q].k >= c.plane_hi) {
                    ok[q] = false;  // weighted and counted, no entries: another rank's plane
                    continue;
                }
                footprint_tiles(c, p[q], p[q].k, t[q]);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (t[q][r] >= 0) slot[q][r] = atomicAdd(cursor + t[q][r] * c.cstride, 1u);
            }
#pragma unroll
            for (int q = 0; q < kVisPerThread; ++q) {
                if (!ok[q]) continue;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (t[q][r] >= 0) {
                        entries[slot[q][r]] = rec[q];
                        ++nent;
                    }
            }
        }
        const float tot = block_sum(sw);
        if (threadIdx.x == 0 && tot != 0.0f) atomicAdd(chan_sw + chan, (double)tot);
    });
    // counters: one set of atomics per block
    __shared__ unsigned s_g[kPrepThreads / 32], s_d[kPrepThreads / 32], s_e[kPrepThreads / 32];
    gridded = warp_sum(gridded);
    dropped = warp_sum(dropped);
    nent = warp_sum(nent);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_g[wid] = gridded;
        s_d[wid] = dropped;
        s_e[wid] = nent;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long g = 0, d = 0, e = 0;
        for (int j = 0; j < kPrepThreads / 32; ++j) {
            g += s_g[j];
            d += s_d[j];
            e += s_e[j];
        }
        if (g) atomicAdd(&ctr->gridded, g);
        if (d) atomicAdd(&ctr->dropped, d);
        if (e) atomicAdd(&ctr->entries, e);
    }
}

// ------------------------------------------------ adjoint: primary-tile sort

// Placement for the adjoint: coordinates and weight only (no visibility value).
__device__ __forceinline__ bool place_coords(const GridCfg& c, const Inputs& in, int64_t i, Place& p, float& wi)
{
    wi = in.wt ? __ldg(in.wt + i) : 1.0f;
    return place(c, __ldg(in.u + i), __ldg(in.v + i), __ldg(in.w + i), p, 0) && isfinite(wi);
}

// Sort key of the adjoint: the tile of the first footprint cell on the
// measurement's plane (Sw = 1) or on the first plane of its w-footprint,
// clamped to the plane range (Sw > 1).
__device__ __forceinline__ int64_t primary_tile(const GridCfg& c, const Place& p)
{
    const int k = p.k < 0 ? 0 : (p.k > c.nw - 1 ? c.nw - 1 : p.k);
    return (int64_t)k * c.ntp + (p.fv >> c.log2T) * c.ntu + (p.fu >> c.log2T);
}

__global__ void __launch_bounds__(kPrepThreads) k_primary_count(GridCfg c, Inputs in, int64_t m,
                                                                uint32_t* __restrict__ counts)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        Place p;
        float wi;
        if (place_coords(c, in, i, p, wi)) atomicAdd(counts + primary_tile(c, p) * c.cstride, 1u);
    }
}

__global__ void __launch_bounds__(kPrepThreads) k_primary_scatter(GridCfg c, Inputs in, int64_t m,
                                                                  uint32_t* __restrict__ cursor,
                                                                  uint32_t* __restrict__ perm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        Place p;
        float wi;
        if (place_coords(c, in, i, p, wi))
            perm[atomicAdd(cursor + primary_tile(c, p) * c.cstride, 1u)] = (uint32_t)i;
    }
}

// Each sorted measurement of planes [k0, k0+nk) gathers its S x S footprint
// of the (forward-transformed) adjoint planes with the gridding taps, times
// its effective weight.  Consecutive threads take consecutive measurements of
// the same tile, so the footprints they read overlap in L1 / L2.
template <int S>
__global__ void __launch_bounds__(kPrepThreads) k_degrid_gather(GridCfg c, const uint32_t* __restrict__ perm,
                                                                const uint32_t* __restrict__ off, int k0, int nk,
                                                                const float2* __restrict__ planes, Inputs in,
                                                                const uint32_t* __restrict__ density,
                                                                float2* __restrict__ grad)
{
    // measurements whose planes reach [k0, k0 + nk): sort key plane in
    // [k0 - Sw + 1, k0 + nk) (a contiguous run of the sorted list)
    const int klo = k0 - (c.Sw - 1) > 0 ? k0 - (c.Sw - 1) : 0;
    const uint32_t b = off[(int64_t)klo * c.ntp], e = off[(int64_t)(k0 + nk) * c.ntp];
    for (int64_t j = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < e;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = perm[j];
        Place p;
        float wi;
        if (!place_coords(c, in, i, p, wi)) continue;  // cannot happen: perm holds placed ones
        if (c.uniform) wi = wi / (float)__ldg(density + (int64_t)nearest_cell(c, p.pv) * c.n + nearest_cell(c, p.pu));
        float gu[S], gv[S];
        eval_taps<S>(c, p.pu, p.fu, gu);
        eval_taps<S>(c, p.pv, p.fv, gv);
        float su = 0.f, sv = 0.f;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            su += gu[t];
            sv += gv[t];
        }
#pragma unroll
        for (int t = 1; t < S; t += 2) {
            gu[t] = -gu[t];
            gv[t] = -gv[t];
        }
        // its planes in this group: the one plane (Sw = 1), or the w-footprint
        // with the normalised w-taps (Sw > 1)
        const float hn = c.Sw > 1 ? w_tap_norm(c, p) : 1.0f;
        float ar = 0.f, ai = 0.f;
        for (int tw = 0; tw < c.Sw; ++tw) {
            const int plane = p.k + tw;
            if (plane < k0 || plane >= k0 + nk) continue;
            const float ht = c.Sw > 1 ? w_kernel(c, __fsub_rn((float)plane, p.pw)) * hn : 1.0f;
            const float2* P = planes + (int64_t)(plane - k0) * c.n * c.n + p.fu;
            float cr = 0.f, ci = 0.f;
#pragma unroll
            for (int rr = 0; rr < S; ++rr) {
                const float2* R = P + (int64_t)plane_row(c, p.fv + rr) * c.n;
                float br = 0.f, bi = 0.f;
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const float2 x = __ldg(R + t);
                    br = fmaf(gu[t], x.x, br);
                    bi = fmaf(gu[t], x.y, bi);
                }
                cr = fmaf(gv[rr], br, cr);
                ci = fmaf(gv[rr], bi, ci);
            }
            ar = fmaf(ht, cr, ar);
            ai = fmaf(ht, ci, ai);
        }
        float scale = wi / (su * sv);
        if ((p.fu + p.fv) & 1) scale = -scale;
        // a mirrored measurement enters as conj(V): its gradient is conjugated
        const float2 gi = make_float2(ar * scale, p.conj ? -ai * scale : ai * scale);
        if (c.Sw == 1) {
            grad[i] = gi;
        } else {  // a w-footprint can span plane groups: add this group's part
            const float2 prev = grad[i];
            grad[i] = make_float2(prev.x + gi.x, prev.y + gi.y);
        }
    }
}

// ------------------------------------------------------------------ scan

// Exclusive scan of one value per thread across a 1024-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const uint32_t prefix = wid ? ws[wid - 1] : 0u;
    *total = ws[31];
    __syncthreads();
    return prefix + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_local(const uint32_t* __restrict__ in, int64_t len,
                                                           int stride, uint32_t* __restrict__ out,
                                                           uint32_t* __restrict__ block_sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t x[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        x[j] = (base + j < len) ? in[(base + j) * stride] : 0u;
        s += x[j];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < len) out[base + j] = run;
        run += x[j];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Exclusive scan of the block totals in place (one block, any length), and
// the grand total into out[len].
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(uint32_t* __restrict__ sums, int64_t nb,
                                                          uint32_t* __restrict__ out, int64_t len)
{
    uint32_t carry = 0;
    for (int64_t s0 = 0; s0 < nb; s0 += kScanBlock) {
        const int64_t i = s0 + threadIdx.x;
        const uint32_t v = (i < nb) ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) out[len] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_add(const uint32_t* __restrict__ sums, int64_t len,
                                                         int stride, uint32_t* __restrict__ out,
                                                         uint32_t* __restrict__ cursor)
{
    const uint32_t add = sums[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < len) {
            const uint32_t o = out[base + j] + add;
            out[base + j] = o;
            cursor[(base + j) * stride] = o;
        }
    }
}

}  // namespace

cudaError_t launch_primary_count(const GridCfg& c, const float* u, const float* v, const float* w,
                                 const float* wt, int64_t m, uint32_t* counts, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_primary_count<<<prep_blocks(m), kPrepThreads, 0, s>>>(c, Inputs{u, v, w, wt, nullptr}, m, counts);
    return cudaGetLastError();
}

cudaError_t launch_primary_scatter(const GridCfg& c, const float* u, const float* v, const float* w,
                                   const float* wt, int64_t m, uint32_t* cursor, uint32_t* perm,
                                   cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_primary_scatter<<<prep_blocks(m), kPrepThreads, 0, s>>>(c, Inputs{u, v, w, wt, nullptr}, m, cursor, perm);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_gather_s(const GridCfg& c, const uint32_t* perm, const uint32_t* off, int k0, int nk,
                            const float2* planes, const Inputs& in, const uint32_t* density, float2* grad,
                            int64_t m, cudaStream_t s)
{
    k_degrid_gather<S><<<prep_blocks(m), kPrepThreads, 0, s>>>(c, perm, off, k0, nk, planes, in, density, grad);
    return cudaGetLastError();
}

cudaError_t launch_degrid_gather(const GridCfg& c, const uint32_t* perm, const uint32_t* offsets, int k0, int nk,
                                 const float2* planes, const float* u, const float* v, const float* w,
                                 const float* wt, const uint32_t* density, float2* grad, cudaStream_t s)
{
    // the launch is sized for the whole input; threads beyond the group's range exit at once
    const Inputs in{u, v, w, wt, nullptr};
    const int64_t m = (int64_t)sm_count() * 8 * kPrepThreads;
    switch (c.S) {
#define RICK_GATHER_CASE(SS) \
    case SS: return launch_gather_s<SS>(c, perm, offsets, k0, nk, planes, in, density, grad, m, s);
        RICK_GATHER_CASE(1) RICK_GATHER_CASE(2) RICK_GATHER_CASE(3) RICK_GATHER_CASE(4)
        RICK_GATHER_CASE(5) RICK_GATHER_CASE(6) RICK_GATHER_CASE(7) RICK_GATHER_CASE(8)
        RICK_GATHER_CASE(9) RICK_GATHER_CASE(10) RICK_GATHER_CASE(11) RICK_GATHER_CASE(12)
        RICK_GATHER_CASE(13) RICK_GATHER_CASE(14) RICK_GATHER_CASE(15) RICK_GATHER_CASE(16)
#undef RICK_GATHER_CASE
        default: return cudaErrorInvalidValue;
    }
}

size_t scan_block_sums_len(int64_t len)
{
    return (size_t)((len + kScanTile - 1) / kScanTile) + 1;
}

cudaError_t launch_density(const GridCfg& c, const float* u, const float* v, const float* w,
                           const float* wt, const float2* vis, int64_t m, uint32_t* density,
                           cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_density<<<prep_blocks(m), kPrepThreads, 0, s>>>(c, Inputs{u, v, w, wt, vis}, m, density);
    return cudaGetLastError();
}

cudaError_t launch_count(const GridCfg& c, const float* u, const float* v, const float* w,
                         const float* wt, const float2* vis, int64_t m, uint32_t* counts,
                         cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_count<<<prep_blocks(m, c.prep_bpsm), kPrepThreads, 0, s>>>(c, Inputs{u, v, w, wt, vis}, m, counts);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* counts, int64_t len, int stride, uint32_t* offsets, uint32_t* cursor,
                        uint32_t* block_sums, cudaStream_t s)
{
    const int64_t nb = (len + kScanTile - 1) / kScanTile;
    if (nb > 0x7fffffff) return cudaErrorInvalidValue;
    if (nb == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
    k_scan_local<<<(unsigned)nb, kScanBlock, 0, s>>>(counts, len, stride, offsets, block_sums);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(block_sums, nb, offsets, len);
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(block_sums, len, stride, offsets, cursor);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const GridCfg& c, const float* u, const float* v, const float* w,
                           const float* wt, const float2* vis, int64_t m, const uint32_t* density,
                           uint32_t* cursor, float4* entries, Counters* ctr, double* chan_sw, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_scatter<<<prep_blocks(m, c.prep_bpsm), kPrepThreads, 0, s>>>(c, Inputs{u, v, w, wt, vis}, m, density, cursor,
                                                      entries, ctr, chan_sw ? chan_sw : &ctr->sum_w);
    return cudaGetLastError();
}

}  // namespace rick
