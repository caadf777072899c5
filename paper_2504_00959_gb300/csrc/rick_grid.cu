// rick_grid.cu -- convolutional gridding, Eq. 3 of the paper (sub-step 2 of
// step 2 in Sec. 2.1).
//
// The counting sort of rick_prep.cu lists every (measurement, tile) pair whose
// S x S footprint touches a T x T tile of a w-plane, with the measurement's
// weighted, tap-normalised visibility.  Here each tile is owned by one warp
// (k_grid_tiles): the warp accumulates its entries into a private copy of the
// tile in shared memory and writes the whole tile once with coalesced 16-byte
// stores -- also when it is empty, so the planes need no memset and HBM sees
// each plane byte once.  No atomics, global or shared:
//   * entries are taken 32 at a time: each lane loads one (a coalesced
//     512-byte load per warp) and evaluates its 2S taps (degree-10
//     polynomials) into a per-warp stage in shared memory;
//   * the warp then walks the 32 staged entries; the S x S footprint is cut
//     into S rows of S/2 + 1 pairs of horizontally adjacent cells aligned to
//     even columns, and every lane owns fixed (row, pair) slots, read and
//     written as one 16-byte value (4 FMAs per slot);
//   * the tile's pitch in pairs is 4 (mod 8), so the 8 lanes of every phase
//     of a 128-bit access (2 rows x 4 pairs) hit 8 different 16-byte bank
//     groups: the read-modify-write of a footprint is conflict-free;
//   * a __syncwarp between entries orders one entry's stores before the next
//     entry's loads.
// Tiles with more than heavy_threshold() entries (the dense centre of the uv
// plane) would serialise on one warp: k_grid_tiles writes them as zeros and
// lists them as chunks of at most that many entries, and k_grid_chunks
// gives every chunk to a warp, which adds its private tile into the plane
// with vector atomic adds.  The fftshift checkerboard (-1)^(ju+jv) is folded
// into the tap signs.
#include "rick_internal.cuh"

namespace rick {
namespace {

// Chunking threshold of a pass with E entries: E / kHeavyDiv clamped to
// [kHeavyMin, kHeavyMax].  A tile of many entries left to k_grid_tiles costs
// its warp time proportional to the entries, run alone if it comes late in
// the launch; a large pass hides that tail and gains from fewer chunk
// flushes, a small one does not.
constexpr uint32_t kHeavyMin = 64;
constexpr uint32_t kHeavyMax = 768;
constexpr uint32_t kHeavyDiv = 16384;
constexpr int kTilesPerWarp = 8;

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

// A shared-memory tile is T rows of cell pairs (16-byte float4 units) with a
// row pitch of P2 >= T/2 pairs, P2 = 4 (mod 8): the 8 lanes of each phase of
// a 128-bit access (2 footprint rows x 4 pairs, or 8 pairs of one row in
// whole-tile passes) then fall in 8 different 16-byte bank groups, and the
// address of footprint slot (sr, sp) of an entry is the entry's base plus a
// per-lane constant.
__host__ __device__ __forceinline__ int pair_pitch(int T)
{
    const int h = T / 2;
    return h + ((4 - h % 8) % 8 + 8) % 8;
}

int light_warps(int T) { return T <= 16 ? 8 : (T <= 32 ? 4 : 1); }

// Per-lane constants: the footprint cells this lane updates for every entry,
// as (row, pair) slots.  A footprint row of S cells starting at column lu
// spans kPairs cell pairs aligned to even tile columns (the first or last
// pair holds one zero tap); slot s of a lane is pair index lane + 32 s of the
// row-major list of (row, pair).  loff is the slot's byte offset from the
// footprint's first pair in the tile.
template <int S>
struct LaneSlots {
    static constexpr int kPairs = S / 2 + 1;
    static constexpr int kSlots = (S * kPairs + 31) / 32;
    int sr[kSlots], sp[kSlots];
    uint32_t loff[kSlots];
    uint32_t lanebit;

    __device__ __forceinline__ void init(int lane, int p2)
    {
        lanebit = 1u << lane;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int i = lane + 32 * s;
            sr[s] = i < S * kPairs ? i / kPairs : 0;
            sp[s] = i < S * kPairs ? i % kPairs : 0;
            loff[s] = (uint32_t)(sr[s] * p2 + sp[s]) * 16u;
        }
    }
};

// Read-modify-write of one tile pair at shared address addr when this lane's
// bit is set in mask: (c0, c1) += (ga, gb) x (vr + i vi).  Shared-window
// addressing keeps the address arithmetic 32-bit; the predicate replaces a
// branch.
__device__ __forceinline__ void rmw_pair(uint32_t addr, uint32_t mask, uint32_t lanebit, float ga, float gb,
                                         float vr, float vi)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b32 t;\n\t.reg .f32 a, b, c, d;\n\t"
        "and.b32 t, %0, %1;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "@p ld.shared.v4.f32 {a, b, c, d}, [%2];\n\t"
        "@p fma.rn.f32 a, %3, %5, a;\n\t"
        "@p fma.rn.f32 b, %3, %6, b;\n\t"
        "@p fma.rn.f32 c, %4, %5, c;\n\t"
        "@p fma.rn.f32 d, %4, %6, d;\n\t"
        "@p st.shared.v4.f32 [%2], {a, b, c, d};\n\t}"
        :
        : "r"(mask), "r"(lanebit), "r"(addr), "f"(ga), "f"(gb), "f"(vr), "f"(vi)
        : "memory");
}

// Per-warp staging of 32 entries in shared memory: each entry's u taps laid
// out on its pair grid (kPairs pairs, zero-padded on the side of the odd
// start column), its v taps times the weighted visibility (complex), and a
// header: the shared address of its first pair, then one word per slot of
// lane bits saying which lanes' pairs lie inside the tile.
template <int S>
struct Stage {
    static constexpr int kPairs = LaneSlots<S>::kPairs;
    static constexpr int kSlots = LaneSlots<S>::kSlots;
    static constexpr int kHead = kSlots + 1 <= 2 ? 2 : (kSlots + 1 <= 4 ? 4 : 8);
    float2 gu[32 * kPairs];
    float2 gvv[32 * S];
    uint32_t head[32 * kHead];
};

// Shared memory of one warp: its tile (T rows of pitch P2 pairs) and its stage.
template <int S>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int T)
{
    return (size_t)T * pair_pitch(T) * sizeof(float4) + sizeof(Stage<S>);
}

// One staged entry in registers: its header, and for each of the lane's
// slots the u tap pair and the complex v tap x visibility.
template <int S>
struct Staged {
    static constexpr int NS = LaneSlots<S>::kSlots, NH = Stage<S>::kHead;
    uint32_t h[NH];
    float2 g2[NS], gq[NS];

    __device__ __forceinline__ void load(const Stage<S>& st, const LaneSlots<S>& ls, int q)
    {
        const uint4* hp = reinterpret_cast<const uint4*>(st.head + q * NH);
        if (NH == 2) {
            const uint2 x = *reinterpret_cast<const uint2*>(st.head + q * NH);
            h[0] = x.x;
            h[1] = x.y;
        } else {
#pragma unroll
            for (int k = 0; k < NH / 4; ++k) {
                const uint4 x = hp[k];
                h[4 * k] = x.x;
                h[4 * k + 1] = x.y;
                h[4 * k + 2] = x.z;
                h[4 * k + 3] = x.w;
            }
        }
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
            g2[sl] = st.gu[q * Stage<S>::kPairs + ls.sp[sl]];
            gq[sl] = st.gvv[q * S + ls.sr[sl]];
        }
    }

    __device__ __forceinline__ void apply(const LaneSlots<S>& ls) const
    {
#pragma unroll
        for (int sl = 0; sl < NS; ++sl)
            rmw_pair(h[0] + ls.loff[sl], h[1 + sl], ls.lanebit, g2[sl].x, g2[sl].y, gq[sl].x, gq[sl].y);
    }
};

// Stage one entry r of the tile at (u0, v0) into slot `slot` of the warp's
// stage: its 2S taps (degree-10 polynomials with uniform coefficients from
// the constant bank, checkerboard signs folded in), the v taps times the
// visibility, and the header (tile_s: the warp's tile copy).
template <int S>
__device__ __forceinline__ void stage_entry(const GridCfg& c, const float4& r, int u0, int v0, Stage<S>& st,
                                            int slot, uint32_t tile_s, int shift)
{
    constexpr int KP = Stage<S>::kPairs, NS = Stage<S>::kSlots, NH = Stage<S>::kHead;
    const int TP = c.T / 2, P2 = pair_pitch(c.T);
    const int fu = first_cell(c, r.x), fv = first_cell(c, r.y);
    const float zu = __fmaf_rn(2.0f, __fsub_rn(__fsub_rn(r.x, c.half_s), (float)(fu - 1)), -1.0f);
    const float zv = __fmaf_rn(2.0f, __fsub_rn(__fsub_rn(r.y, c.half_s), (float)(fv - 1)), -1.0f);
    const int lu = fu - u0, lv = fv - v0;
    const int odd = lu & 1;  // u0 is even: the parity of the tile column
    const int pu = (lu - odd) / 2;
    float gu[S];
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
        gu[t] = a;
        st.gvv[slot * S + t] = make_float2(bb * r.z, bb * r.w);
    }
    // pair t holds tile columns 2 (pu + t) and 2 (pu + t) + 1: taps
    // (2t, 2t+1) for an even start column, (2t-1, 2t) for an odd one
#pragma unroll
    for (int t = 0; t < KP; ++t) {
        const float e0 = 2 * t < S ? gu[2 * t < S ? 2 * t : 0] : 0.0f;
        const float e1 = 2 * t + 1 < S ? gu[2 * t + 1 < S ? 2 * t + 1 : 0] : 0.0f;
        const float o0 = 2 * t - 1 >= 0 ? gu[2 * t - 1 >= 0 ? 2 * t - 1 : 0] : 0.0f;
        st.gu[slot * KP + t] = odd ? make_float2(o0, e0) : make_float2(e0, e1);
    }
    // header: first pair's shared address (wraps for footprints that start
    // left of or above the tile; only in-tile pairs are used) and the in-tile
    // lane bits of every slot: footprint rows [rlo, rhi) and pairs [plo, phi)
    // lie inside the tile
    const int rlo = max(0, -lv), rhi = min(S, c.T - lv);
    const int plo = max(0, -pu), phi = min(KP, TP - pu);
    const uint32_t pm = phi > plo ? (((1u << phi) - 1u) & ~((1u << plo) - 1u)) : 0u;
    uint32_t wm[NH - 1];
#pragma unroll
    for (int k = 0; k < NH - 1; ++k) wm[k] = 0u;
#pragma unroll
    for (int sr = 0; sr < S; ++sr) {
        const uint32_t rowbits = (sr >= rlo && sr < rhi) ? pm : 0u;
        const int bit = sr * KP, wd = bit / 32, sh = bit % 32;
        wm[wd] |= rowbits << sh;
        if (sh + KP > 32 && wd + 1 < NS) wm[wd + 1] |= rowbits >> (32 - sh);
    }
    st.head[slot * NH] = tile_s + (uint32_t)(lv * P2 + pu) * 16u;
#pragma unroll
    for (int k = 0; k < NH - 1; ++k) st.head[slot * NH + 1 + k] = wm[k];
}

// Walk the staged entries q0 .. q1-1 into the warp's tile: the next entry's
// header and taps are loaded before this entry's read-modify-write (two
// register sets, alternating); a __syncwarp orders consecutive entries.
template <int S>
__device__ __forceinline__ void walk_staged(const Stage<S>& st, const LaneSlots<S>& ls, int q0, int q1)
{
    if (q1 <= q0) return;
    Staged<S> A, B;
    A.load(st, ls, q0);
    for (int q = q0;; q += 2) {
        if (q + 1 < q1) B.load(st, ls, q + 1);
        A.apply(ls);
        __syncwarp();
        if (q + 1 >= q1) break;
        if (q + 2 < q1) A.load(st, ls, q + 2);
        B.apply(ls);
        __syncwarp();
        if (q + 2 >= q1) break;
    }
}

// Accumulate entries [b, e) of one sorted list into the warp's tile.  Rounds
// of 32 entries: (1) each lane takes one entry (coalesced 16-byte loads) and
// evaluates its 2S taps (degree-10 polynomials with uniform coefficients from
// the constant bank) with the checkerboard signs folded in, and its header,
// into the stage (stage_entry); (2) the warp walks the 32 entries; every lane
// updates its slots, each a pair of horizontally adjacent cells read and
// written as one 16-byte value (4 FMAs: u tap pair x complex v
// tap-visibility product).  Within one entry the lanes' pairs are distinct
// and conflict-free.  The stage is read-only during the walk.
template <int S>
__device__ __forceinline__ void warp_grid_range(const GridCfg& c, const float4* __restrict__ ent, uint32_t b,
                                                uint32_t e, int u0, int v0, float4* tile4, Stage<S>& st,
                                                const LaneSlots<S>& ls, int lane, int shift)
{
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile4);
    // each round's entries are loaded one round ahead
    float4 r_next = make_float4(0.f, 0.f, 0.f, 0.f);
    if (b + lane < e) r_next = __ldg(ent + b + lane);
    for (uint32_t j0 = b; j0 < e; j0 += 32) {
        const uint32_t j = j0 + lane;
        const float4 r = r_next;
        if (j + 32 < e) r_next = __ldg(ent + j + 32);
        if (j < e) stage_entry<S>(c, r, u0, v0, st, lane, tile_s, shift);
        __syncwarp();
        walk_staged<S>(st, ls, 0, (e - j0 < 32u) ? (int)(e - j0) : 32);
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
    int rem, tv, tu;
    if (c.ntu_log2 >= 0) {
        // power-of-two tiles per side: shifts instead of 64-bit division
        g.kl = (int)(tl >> (2 * c.ntu_log2));
        rem = (int)(tl & (c.ntp - 1));
        tv = rem >> c.ntu_log2;
        tu = rem & (c.ntu - 1);
    } else {
        g.kl = (int)(tl / c.ntp);
        rem = (int)(tl - (int64_t)g.kl * c.ntp);
        tv = rem / c.ntu;
        tu = rem - tv * c.ntu;
    }
    g.tg = (int64_t)(k0 + g.kl) * c.ntp + rem;
    g.u0 = tu * c.T;
    g.v0 = tv * c.T;
    g.wu = min(c.T, c.n - g.u0);
    g.wv = min(c.T, c.n - g.v0);
    return g;
}

// Whole-tile passes of one warp: lane L keeps the pair column L mod (T/2)
// and starts at row L / (T/2), stepping 32 / (T/2) rows, so every pass is a
// run of 16-byte accesses with no division.  The pair of grid row v0 + row
// is at plane_row(v0 + row) n + u0 + 2 pr, 16-byte aligned because n and u0
// are even.
struct TileWalk {
    int pr, r0, dr, p2;
};

__device__ __forceinline__ TileWalk tile_walk(const GridCfg& c, int lane)
{
    TileWalk w;
    const int ltp = c.log2T - 1;
    w.p2 = pair_pitch(c.T);
    w.pr = lane & ((1 << ltp) - 1);
    w.r0 = lane >> ltp;
    w.dr = 32 >> ltp;
    return w;
}

// The walk's rows r0, r0 + dr, ... in runs: within 16 grid rows starting at
// a multiple of 16 (v0 is one), consecutive rows of the walk are dr memory
// rows apart with natural rows and dr N1 apart in b-major order, so each run
// advances one pointer by a constant (no per-row plane_row); natural rows
// make one run of the whole tile.
__device__ __forceinline__ int64_t walk_mem_step(const GridCfg& c, const TileWalk& w)
{
    return (int64_t)w.dr * (c.row_perm ? (c.n >> 4) : 1) * (c.n / 2);  // in float4 (cell pair) units
}

// Write the valid part of a tile to the plane (or zeros): coalesced 16-byte
// stores, 256 contiguous bytes per row segment for T = 32.
template <bool kZero>
__device__ __forceinline__ void store_tile(const GridCfg& c, const TileGeom& g, float2* P0, const float4* tile4,
                                           int lane)
{
    const TileWalk w = tile_walk(c, lane);
    if (2 * w.pr >= g.wu) return;
    float2* col = P0 + g.u0 + 2 * w.pr;
    const int64_t step = walk_mem_step(c, w);
    for (int row = w.r0; row < g.wv;) {
        const int end = c.row_perm ? min(g.wv, (row | 15) + 1) : g.wv;
        float4* dst = reinterpret_cast<float4*>(col + (int64_t)plane_row(c, g.v0 + row) * c.n);
#pragma unroll 4
        for (; row < end; row += w.dr, dst += step)
            *dst = kZero ? make_float4(0.f, 0.f, 0.f, 0.f) : tile4[row * w.p2 + w.pr];
    }
}

// Initialise a tile copy: zeros, or the plane's current values (accumulating
// pass; cells outside the grid start at zero).
__device__ __forceinline__ void init_tile(const GridCfg& c, const TileGeom& g, const float2* P0, float4* tile4,
                                          bool from_plane, int lane)
{
    const TileWalk w = tile_walk(c, lane);
    if (!from_plane || 2 * w.pr >= g.wu) {
#pragma unroll 4
        for (int row = w.r0; row < c.T; row += w.dr) tile4[row * w.p2 + w.pr] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float2* col = P0 + g.u0 + 2 * w.pr;
    const int64_t step = walk_mem_step(c, w);
    for (int row = w.r0; row < c.T;) {
        const int end = c.row_perm ? min(c.T, (row | 15) + 1) : c.T;
        const float4* src = reinterpret_cast<const float4*>(col + (int64_t)plane_row(c, g.v0 + row) * c.n);
#pragma unroll 4
        for (; row < end; row += w.dr, src += step)
            tile4[row * w.p2 + w.pr] = row < g.wv ? *src : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Chunking threshold of the pass [k0, k0 + ntl / ntp) from its entry count
// (the offsets the gridder reads anyway: tile k0 * ntp + ntl is the end of
// the last tile's range).  Both gridder kernels derive the same value.  A
// pass over several entry lists is never chunked.
__device__ __forceinline__ uint32_t heavy_threshold(const GridCfg& c, const ChunkList& ch, int k0, int64_t ntl)
{
    if (ch.count != 1) return 0xffffffffu;
    const int64_t t0 = (int64_t)k0 * c.ntp;
    const uint32_t entries = __ldg(ch.off[0] + t0 + ntl) - __ldg(ch.off[0] + t0);
    return min(max(entries / kHeavyDiv, kHeavyMin), kHeavyMax);
}

// Each CTA of W warps takes kTilesPerWarp * W consecutive tiles of the pass,
// warp w the tiles w, w + W, ... of them (neighbours, so similar loads), and
// loads the next tile's list ranges while it grids the current one; the
// hardware hands CTAs out dynamically, which balances the uneven tiles.
// Lane q < ch.count holds the range of list q for the tile.
template <int S>
__global__ void __launch_bounds__(256, S <= 8 ? 2 : 0) k_grid_tiles(GridCfg c, ChunkList ch, int k0, int64_t ntl,
                                                                   int shift,
                                                    int accumulate, float2* __restrict__ planes,
                                                    uint32_t* __restrict__ heavy_list, uint32_t heavy_cap)
{
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwt = blockDim.x >> 5;
    const int64_t first = (int64_t)blockIdx.x * nwt * kTilesPerWarp;
    const int64_t last = min(ntl, first + nwt * kTilesPerWarp);
    int64_t tl = first + wid;
    if (tl >= last) return;
    const uint32_t heavy = heavy_threshold(c, ch, k0, ntl);
    unsigned char* mine = reinterpret_cast<unsigned char*>(smem4) + (size_t)wid * warp_smem_bytes<S>(c.T);
    float4* tile4 = reinterpret_cast<float4*>(mine);
    Stage<S>& st = *reinterpret_cast<Stage<S>*>(mine + (size_t)c.T * pair_pitch(c.T) * sizeof(float4));
    LaneSlots<S> ls;
    ls.init(lane, pair_pitch(c.T));

    if constexpr (S <= 8) if (ch.count == 1) {
        // One list: the warp's tiles tl + k nwt (k < kTilesPerWarp), lane k
        // holding tile k's range.  Consecutive tiles with at most 32 entries
        // in all share one staging round (the taps of a light tile's few
        // entries would otherwise cost a whole round of polynomial
        // evaluations); each is then initialised, walked over its slots of
        // the stage and stored in turn.  Heavier tiles take rounds of their
        // own, the heaviest go to k_grid_chunks.  (Supports up to 8: wider
        // footprints keep the registers of the tile-by-tile loop below.)
        const uint32_t full = 0xffffffffu;
        const int64_t tk = tl + (int64_t)lane * nwt;
        uint32_t rb = 0, rn = 0;
        if (lane < kTilesPerWarp && tk < last) {
            const int64_t tg = (int64_t)k0 * c.ntp + tk;
            rb = __ldg(ch.off[0] + tg);
            rn = __ldg(ch.off[0] + tg + 1) - rb;
        }
        const int ntw = (int)min((int64_t)kTilesPerWarp, (last - tl + nwt - 1) / nwt);
        const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile4);
        for (int k = 0; k < ntw;) {
            const uint32_t nk = __shfl_sync(full, rn, k);
            if (nk > 32u) {
                const int64_t tlk = tl + (int64_t)k * nwt;
                const uint32_t bk = __shfl_sync(full, rb, k);
                ++k;
                const TileGeom g = tile_geom(c, k0, tlk);
                float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
                if (nk > heavy) {
                    // hand the tile to k_grid_chunks as chunks of at most
                    // `heavy` entries, which add into the plane; the tile
                    // starts at zero unless this pass accumulates
                    const uint32_t nchunks = (nk + heavy - 1) / heavy;
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(heavy_list, nchunks);
                    base = __shfl_sync(full, base, 0);
                    if (base + nchunks <= heavy_cap) {
                        for (uint32_t q = lane; q < nchunks; q += 32) {
                            heavy_list[1 + 2 * (base + q)] = (uint32_t)tlk;
                            heavy_list[2 + 2 * (base + q)] = q;
                        }
                        if (!accumulate) store_tile<true>(c, g, P0, nullptr, lane);
                        continue;
                    }
                    // no room in the chunk list: mark the reserved slots that
                    // do exist as empty, and grid the tile here
                    for (uint32_t q = base + lane; q < heavy_cap; q += 32) heavy_list[1 + 2 * q] = 0xffffffffu;
                }
                init_tile(c, g, P0, tile4, accumulate != 0, lane);
                __syncwarp();
                warp_grid_range<S>(c, ch.ent[0], bk, bk + nk, g.u0, g.v0, tile4, st, ls, lane, shift);
                __syncwarp();
                store_tile<false>(c, g, P0, tile4, lane);
                __syncwarp();
                continue;
            }
            // the run of tiles k .. k+m-1 with at most 32 entries in all
            int m = 0;
            uint32_t tot = 0;
            while (k + m < ntw) {
                const uint32_t cm = __shfl_sync(full, rn, k + m);
                if (tot + cm > 32u) break;
                tot += cm;
                ++m;
            }
            if (tot > 0) {
                // lane j < tot stages entry j of the run (of tile k + ij)
                uint32_t pre = 0, bj = 0;
                int ij = 0;
                for (int q = 0; q < m; ++q) {
                    const uint32_t cq = __shfl_sync(full, rn, k + q), bq = __shfl_sync(full, rb, k + q);
                    if ((uint32_t)lane >= pre && (uint32_t)lane < pre + cq) {
                        ij = q;
                        bj = bq + ((uint32_t)lane - pre);
                    }
                    pre += cq;
                }
                if ((uint32_t)lane < tot) {
                    const TileGeom gj = tile_geom(c, k0, tl + (int64_t)(k + ij) * nwt);
                    stage_entry<S>(c, __ldg(ch.ent[0] + bj), gj.u0, gj.v0, st, lane, tile_s, shift);
                }
                __syncwarp();
            }
            uint32_t pre = 0;
            for (int q = 0; q < m; ++q) {
                const uint32_t cq = __shfl_sync(full, rn, k + q);
                const TileGeom g = tile_geom(c, k0, tl + (int64_t)(k + q) * nwt);
                float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
                if (cq == 0) {
                    if (!accumulate) store_tile<true>(c, g, P0, nullptr, lane);
                    continue;
                }
                init_tile(c, g, P0, tile4, accumulate != 0, lane);
                __syncwarp();
                walk_staged<S>(st, ls, (int)pre, (int)(pre + cq));
                __syncwarp();
                store_tile<false>(c, g, P0, tile4, lane);
                __syncwarp();  // the next tile's init overwrites the tile copy
                pre += cq;
            }
            k += m;
        }
        return;
    }

    // several lists (a pass over more than one chunk of entries): tile by tile
    auto fetch = [&](int64_t t, uint32_t& rb, uint32_t& re) {
        rb = re = 0;
        if (t < last && lane < ch.count) {
            const int64_t tg = (int64_t)k0 * c.ntp + t;
            rb = __ldg(ch.off[lane] + tg);
            re = __ldg(ch.off[lane] + tg + 1);
        }
    };
    uint32_t nb, ne;
    fetch(tl, nb, ne);
    for (; tl < last; tl += nwt) {
        const uint32_t cb = nb, ce = ne;
        fetch(tl + nwt, nb, ne);
        const TileGeom g = tile_geom(c, k0, tl);
        float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
        uint32_t nent = ce - cb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nent += __shfl_xor_sync(0xffffffffu, nent, o);

        if (nent > heavy && ch.count == 1) {
            // many entries: hand the tile to k_grid_chunks as chunks of at most
            // `heavy` entries, which add into the plane; the tile starts at
            // zero unless this pass accumulates onto earlier chunks
            const uint32_t nchunks = (nent + heavy - 1) / heavy;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(heavy_list, nchunks);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + nchunks <= heavy_cap) {
                for (uint32_t k = lane; k < nchunks; k += 32) {
                    heavy_list[1 + 2 * (base + k)] = (uint32_t)tl;
                    heavy_list[2 + 2 * (base + k)] = k;
                }
                if (!accumulate) store_tile<true>(c, g, P0, nullptr, lane);
                continue;
            }
            // no room in the chunk list: mark the reserved slots that do exist
            // as empty, and grid the tile here (correct, slower)
            for (uint32_t k = base + lane; k < heavy_cap; k += 32) heavy_list[1 + 2 * k] = 0xffffffffu;
        }
        if (nent == 0) {
            if (!accumulate) store_tile<true>(c, g, P0, nullptr, lane);
            continue;
        }
        init_tile(c, g, P0, tile4, accumulate != 0, lane);
        __syncwarp();
        for (int q = 0; q < ch.count; ++q) {
            const uint32_t b = __shfl_sync(0xffffffffu, cb, q), e = __shfl_sync(0xffffffffu, ce, q);
            if (e > b) warp_grid_range<S>(c, ch.ent[q], b, e, g.u0, g.v0, tile4, st, ls, lane, shift);
        }
        __syncwarp();
        store_tile<false>(c, g, P0, tile4, lane);
        __syncwarp();  // the next tile's init overwrites the tile copy
    }
}

// Chunks of the tiles with many entries: one warp per chunk, private tile in
// shared memory, flushed into the plane with 16-byte vector atomic adds of
// the non-zero cell pairs (the tile's cells were zeroed by k_grid_tiles,
// which ran before on the same stream).
template <int S>
__global__ void __launch_bounds__(256) k_grid_chunks(GridCfg c, ChunkList ch, int k0, int64_t ntl, int shift,
                                                     float2* __restrict__ planes,
                                                     const uint32_t* __restrict__ heavy_list, uint32_t heavy_cap)
{
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* mine = reinterpret_cast<unsigned char*>(smem4) + (size_t)wid * warp_smem_bytes<S>(c.T);
    float4* tile4 = reinterpret_cast<float4*>(mine);
    Stage<S>& st = *reinterpret_cast<Stage<S>*>(mine + (size_t)c.T * pair_pitch(c.T) * sizeof(float4));
    LaneSlots<S> ls;
    ls.init(lane, pair_pitch(c.T));
    const uint32_t heavy = heavy_threshold(c, ch, k0, ntl);
    const uint32_t count = min(heavy_list[0], heavy_cap);
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t it = blockIdx.x * (blockDim.x >> 5) + wid; it < count; it += nwarps) {
        const uint32_t tl32 = heavy_list[1 + 2 * it];
        if (tl32 == 0xffffffffu) continue;  // slot of a tile gridded by k_grid_tiles itself
        const int64_t tl = tl32;
        const uint32_t k = heavy_list[2 + 2 * it];
        const TileGeom g = tile_geom(c, k0, tl);
        float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
        const uint32_t b0 = ch.off[0][g.tg], e0 = ch.off[0][g.tg + 1];
        const uint32_t b = b0 + k * heavy;
        const uint32_t e = min(e0, b + heavy);
        init_tile(c, g, P0, tile4, false, lane);
        __syncwarp();
        warp_grid_range<S>(c, ch.ent[0], b, e, g.u0, g.v0, tile4, st, ls, lane, shift);
        __syncwarp();
        const TileWalk w = tile_walk(c, lane);
        if (2 * w.pr < g.wu) {
            float2* col = P0 + g.u0 + 2 * w.pr;
            const int64_t step = walk_mem_step(c, w);
            for (int row = w.r0; row < g.wv;) {
                const int end = c.row_perm ? min(g.wv, (row | 15) + 1) : g.wv;
                float4* dst = reinterpret_cast<float4*>(col + (int64_t)plane_row(c, g.v0 + row) * c.n);
                for (; row < end; row += w.dr, dst += step) {
                    const float4 x = tile4[row * w.p2 + w.pr];
                    if (x.x != 0.f || x.y != 0.f || x.z != 0.f || x.w != 0.f) atomicAdd(dst, x);
                }
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
                          float2* planes, uint32_t* heavy, size_t heavy_words, cudaStream_t s)
{
    const int64_t ntl = (int64_t)nk * c.ntp;
    if (ntl <= 0) return cudaSuccess;
    const size_t tile_bytes = warp_smem_bytes<S>(c.T);
    const int wl = light_warps(c.T);
    const int64_t nblocks = (ntl + wl - 1) / wl;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    // heavy: [count, (tile, chunk) pairs]
    const size_t pairs = (heavy_words - 1) / 2;
    const uint32_t cap = (uint32_t)(pairs < 0x7fffffffu ? pairs : 0x7fffffffu);
    cudaError_t e = cudaMemsetAsync(heavy, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if ((e = allow_smem(k_grid_tiles<S>, tile_bytes * wl)) != cudaSuccess) return e;
    if ((e = allow_smem(k_grid_chunks<S>, tile_bytes * wl)) != cudaSuccess) return e;
    const unsigned tile_blocks = (unsigned)((nblocks + kTilesPerWarp - 1) / kTilesPerWarp);
    k_grid_tiles<S><<<tile_blocks, 32 * wl, tile_bytes * wl, s>>>(c, ch, k0, ntl, shift ? 1 : 0, accumulate ? 1 : 0,
                                                                  planes, heavy, cap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_chunks<S>, 32 * wl, tile_bytes * wl)) !=
        cudaSuccess)
        return e;
    const unsigned nchunk_blocks = (unsigned)(max(per_sm, 1) * sm_count_grid());
    k_grid_chunks<S><<<nchunk_blocks, 32 * wl, tile_bytes * wl, s>>>(c, ch, k0, ntl, shift ? 1 : 0, planes, heavy,
                                                                    cap);
    return cudaGetLastError();
}

}  // namespace

// Every chunk holds more than h / 2 entries on average for a threshold h
// (a heavy tile of n > h entries makes ceil(n / h) < 2 n / h chunks), so a
// pass over E entries lists fewer than 2 E / h <= 2 E / kHeavyMin chunks.
size_t heavy_words_for(int64_t max_entries)
{
    const int64_t chunks = 2 * max_entries / kHeavyMin + 1;
    return 1 + 2 * (size_t)(chunks > 0 ? chunks : 1);
}

cudaError_t launch_grid(const GridCfg& c, const ChunkList& ch, int k0, int nk, bool shift_sign,
                        bool accumulate, uint32_t* heavy, size_t heavy_words, float2* planes, cudaStream_t s)
{
    if (!heavy || heavy_words < 1) return cudaErrorInvalidValue;
    switch (c.S) {
#define RICK_GRID_CASE(SS) \
    case SS: return launch_grid_s<SS>(c, ch, k0, nk, shift_sign, accumulate, planes, heavy, heavy_words, s);
        RICK_GRID_CASE(1) RICK_GRID_CASE(2) RICK_GRID_CASE(3) RICK_GRID_CASE(4)
        RICK_GRID_CASE(5) RICK_GRID_CASE(6) RICK_GRID_CASE(7) RICK_GRID_CASE(8)
        RICK_GRID_CASE(9) RICK_GRID_CASE(10) RICK_GRID_CASE(11) RICK_GRID_CASE(12)
        RICK_GRID_CASE(13) RICK_GRID_CASE(14) RICK_GRID_CASE(15) RICK_GRID_CASE(16)
#undef RICK_GRID_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rick
