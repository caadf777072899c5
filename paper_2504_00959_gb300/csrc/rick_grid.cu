// rick_grid.cu -- convolutional gridding, Eq. 3 of the paper (sub-step 2 of
// step 2 in Sec. 2.1).
//
// The counting sort of rick_prep.cu lists every (measurement, tile) pair whose
// S x S footprint touches a T x T tile of a w-plane, with the measurement's
// weighted, tap-normalised visibility.  Here each tile is owned by one warp
// (k_grid_tiles): the warp accumulates its entries into a private copy of the
// tile in shared memory and writes the whole tile once with coalesced 16-byte
// stores -- also when it is empty, so the planes need no memset and HBM sees
// each plane byte once.  No atomics on the tiles, global or shared:
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
// plane) would serialise on one warp: k_grid_tiles lists them (list counters
// are the only global atomics) and leaves them unwritten.  k_grid_heavy gives
// each one CTA whose warps grid shares of its entries into private copies,
// sums the copies in shared memory and writes the tile once; the 2 CTAs of a
// thread-block cluster share each of the few huge ones and sum their copies
// through distributed shared memory.  The fftshift checkerboard (-1)^(ju+jv)
// is folded into the tap signs.
#include <algorithm>
#include <atomic>

#include "rick_internal.cuh"

namespace rick {
namespace {

// Heavy-tile threshold of a pass with E entries: E / kHeavyDiv clamped to
// [kHeavyMin, kHeavyMax].  A tile of many entries left to k_grid_tiles costs
// its warp time proportional to the entries, run alone if it comes late in
// the launch; a large pass hides that tail and sends fewer tiles through
// k_grid_heavy's summing of copies, a small one does not.
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
//   TM (tap-major, the tiles kernel): taps stored with a pitch of 33
// entries, so that a staging lane's stores of one tap index are consecutive
// across the warp and a walking warp's reads of one entry (its lanes'
// different tap indices, 66 words apart) fall in different banks; entry-major
// (the heavy-tile kernel) keeps an entry's taps together, which its long
// walks over full rounds execute in fewer instructions.
template <int S, bool TM = true>
struct alignas(16) Stage {
    static constexpr int kPairs = LaneSlots<S>::kPairs;
    static constexpr int kSlots = LaneSlots<S>::kSlots;
    static constexpr int kHead = kSlots + 1 <= 2 ? 2 : (kSlots + 1 <= 4 ? 4 : 8);
    static constexpr int kPitch = 33;
    uint32_t head[32 * kHead];
    float2 gu[kPitch * kPairs];
    float2 gvv[kPitch * S];
    // tap t of staged entry e
    static __device__ __forceinline__ int gu_at(int e, int t) { return TM ? t * kPitch + e : e * kPairs + t; }
    static __device__ __forceinline__ int gvv_at(int e, int t) { return TM ? t * kPitch + e : e * S + t; }
};

// Shared memory of one warp: its tile (T rows of pitch P2 pairs) and its stage.
template <int S>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int T)
{
    return (size_t)T * pair_pitch(T) * sizeof(float4) + sizeof(Stage<S>);
}

// One staged entry in registers: its header, and for each of the lane's
// slots the u tap pair and the complex v tap x visibility.
template <int S, bool TM = true>
struct Staged {
    static constexpr int NS = LaneSlots<S>::kSlots, NH = Stage<S>::kHead;
    uint32_t h[NH];
    float2 g2[NS], gq[NS];

    __device__ __forceinline__ void load(const Stage<S, TM>& st, const LaneSlots<S>& ls, int q)
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
            g2[sl] = st.gu[Stage<S, TM>::gu_at(q, ls.sp[sl])];
            gq[sl] = st.gvv[Stage<S, TM>::gvv_at(q, ls.sr[sl])];
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
template <int S, bool TM = true>
__device__ __forceinline__ void stage_entry(const GridCfg& c, const float4& r, int u0, int v0, Stage<S, TM>& st,
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
        st.gvv[Stage<S, TM>::gvv_at(slot, t)] = make_float2(bb * r.z, bb * r.w);
    }
    // pair t holds tile columns 2 (pu + t) and 2 (pu + t) + 1: taps
    // (2t, 2t+1) for an even start column, (2t-1, 2t) for an odd one
#pragma unroll
    for (int t = 0; t < KP; ++t) {
        const float e0 = 2 * t < S ? gu[2 * t < S ? 2 * t : 0] : 0.0f;
        const float e1 = 2 * t + 1 < S ? gu[2 * t + 1 < S ? 2 * t + 1 : 0] : 0.0f;
        const float o0 = 2 * t - 1 >= 0 ? gu[2 * t - 1 >= 0 ? 2 * t - 1 : 0] : 0.0f;
        st.gu[Stage<S, TM>::gu_at(slot, t)] = odd ? make_float2(o0, e0) : make_float2(e0, e1);
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
template <int S, bool TM = true>
__device__ __forceinline__ void walk_staged(const Stage<S, TM>& st, const LaneSlots<S>& ls, int q0, int q1)
{
    if (q1 <= q0) return;
    Staged<S, TM> A, B;
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
template <int S, bool TM = true>
__device__ __forceinline__ void warp_grid_range(const GridCfg& c, const float4* __restrict__ ent, uint32_t b,
                                                uint32_t e, int u0, int v0, float4* tile4, Stage<S, TM>& st,
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
        if (j < e) stage_entry<S, TM>(c, r, u0, v0, st, lane, tile_s, shift);
        __syncwarp();
        walk_staged<S, TM>(st, ls, 0, (e - j0 < 32u) ? (int)(e - j0) : 32);
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

// Heavy-tile threshold of the pass [k0, k0 + ntl / ntp) from its entry count
// (the offsets the gridder reads anyway: tile k0 * ntp + ntl is the end of
// the last tile's range).  A pass over several entry lists lists no heavy
// tiles.
__device__ __forceinline__ uint32_t heavy_threshold(const GridCfg& c, const ChunkList& ch, int k0, int64_t ntl)
{
    if (ch.count != 1) return 0xffffffffu;
    const int64_t t0 = (int64_t)k0 * c.ntp;
    const uint32_t entries = __ldg(ch.off[0] + t0 + ntl) - __ldg(ch.off[0] + t0);
    return min(max(entries / kHeavyDiv, kHeavyMin), kHeavyMax);
}

// The heavy-tile lists of a pass in one scratch array: w[0] / w[1] count and
// claim the tiles of k_grid_heavy's per-CTA list (slots w[4 ..]), w[2] / w[3]
// those of its per-cluster list of huge tiles (slots w[4 + cap_h ..]).
// Tiles with more than `huge` entries go to the second list while it has room.
struct HeavyList {
    uint32_t* w;
    uint32_t cap_h, cap_x, huge;
};

// List tile `tile` of n entries (warp-uniform call); false when both lists
// are full, and the warp grids the tile itself.
__device__ __forceinline__ bool list_heavy(const HeavyList& hl, uint32_t n, uint32_t tile, int lane)
{
    uint32_t ok = 0;
    if (lane == 0) {
        if (n > hl.huge) {
            const uint32_t slot = atomicAdd(hl.w + 2, 1u);
            if (slot < hl.cap_x) {
                hl.w[4 + hl.cap_h + slot] = tile;
                ok = 1;
            }
        }
        if (!ok) {
            const uint32_t slot = atomicAdd(hl.w, 1u);
            if (slot < hl.cap_h) {
                hl.w[4 + slot] = tile;
                ok = 1;
            }
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Each CTA of W warps takes kTilesPerWarp * W consecutive tiles of the pass,
// warp w the tiles w, w + W, ... of them (neighbours, so similar loads), and
// loads the next tile's list ranges while it grids the current one; the
// hardware hands CTAs out dynamically, which balances the uneven tiles.
// Lane q < ch.count holds the range of list q for the tile.
template <int S>
__global__ void __launch_bounds__(256, S <= 8 ? 2 : 0) k_grid_tiles(GridCfg c, ChunkList ch, int k0, int64_t ntl,
                                                                   int shift,
                                                    int accumulate, float2* __restrict__ planes, HeavyList hl)
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
        // own, the heaviest go to k_grid_heavy.  (Supports up to 8: wider
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
                // list the tile for k_grid_heavy, which writes all of it; with
                // no room left in the lists, grid it here
                if (nk > heavy && list_heavy(hl, nk, (uint32_t)tlk, lane)) continue;
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

        // many entries: list the tile for k_grid_heavy, which writes all of
        // it; with no room left in the lists, grid it here (correct, slower)
        if (nent > heavy && ch.count == 1 && list_heavy(hl, nent, (uint32_t)tl, lane)) continue;
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

// Shared memory of a k_grid_heavy CTA: as many warps (each with a private
// tile copy and a stage) as fit in kHeavySmem, at most kHeavyWarpsMax and at
// least one; two such CTAs share an SM.  A heavy tile gives each warp at least
// kHeavyPerWarp entries (fewer warps on lighter tiles: every active warp's copy
// is summed at the end).  A tile with more than kHugePerWarp entries per warp
// of one CTA is shared by the kHugeCluster CTAs of a cluster, whose warps then
// still take at least 8 rounds of 32 entries each.  Clusters of two CTAs
// fill every CTA slot of the SMs (larger clusters leave slots unused where
// the SMs' CTA slots do not divide into whole clusters: measured on a dense
// 2048^2 x 16-plane channel of 2e7 measurements, 1.45 ms gridding with pairs,
// 1.48 ms with 4 CTAs, 1.49 ms with 8); 512 rather than 2048 entries per warp
// shortens the few longest tiles (64-channel loop 32.6 -> 31.2 ms gridding).
constexpr size_t kHeavySmem = 110 * 1024;
constexpr int kHeavyWarpsMax = 8;
constexpr uint32_t kHeavyPerWarp = 64;
constexpr uint32_t kHugePerWarp = 512;
constexpr int kHugeCluster = 2;

template <int S>
int heavy_warps(int T)
{
    const int w = (int)(kHeavySmem / warp_smem_bytes<S>(T));
    return w < 1 ? 1 : (w > kHeavyWarpsMax ? kHeavyWarpsMax : w);
}

// Thread-block cluster primitives (PTX ISA: %cluster_ctarank, barrier.cluster,
// mapa, ld.shared::cluster).  cluster_sync is the cluster-wide counterpart of
// __syncthreads, with release / acquire ordering of shared-memory accesses.
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of shared address `addr` in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void add4(float4& a, const float4& x)
{
    a.x += x.x;
    a.y += x.y;
    a.z += x.z;
    a.w += x.w;
}

// Per-thread view of a heavy-tile CTA's shared memory: warp wid's tile copy
// and stage, and the constants of the copy-summing loops.
template <int S>
struct HeavyCta {
    float4* tile4;
    Stage<S, false>* st;  // entry-major (both layouts take the same space)
    LaneSlots<S> ls;
    int p2, ltp, pmask, wstride;

    __device__ __forceinline__ HeavyCta(const GridCfg& c, float4* smem4, int wid, int lane)
    {
        const size_t wbytes = warp_smem_bytes<S>(c.T);
        unsigned char* mine = reinterpret_cast<unsigned char*>(smem4) + (size_t)wid * wbytes;
        tile4 = reinterpret_cast<float4*>(mine);
        st = reinterpret_cast<Stage<S, false>*>(mine + (size_t)c.T * pair_pitch(c.T) * sizeof(float4));
        p2 = pair_pitch(c.T);
        ls.init(lane, p2);
        ltp = c.log2T - 1;
        pmask = (1 << ltp) - 1;
        wstride = (int)(wbytes / sizeof(float4));  // a Stage is a multiple of 16 bytes
    }

    // warp `part` of `parts` grids its share of the entries [b0, e0) (whole
    // 32-entry rounds) into its zeroed copy
    __device__ __forceinline__ void grid_share(const GridCfg& c, const ChunkList& ch, const TileGeom& g, uint32_t b0,
                                               uint32_t e0, uint32_t part, uint32_t parts, int lane, int shift)
    {
        const uint32_t rounds = (e0 - b0 + 31) / 32;
        const uint32_t b = b0 + 32 * (uint32_t)(((uint64_t)rounds * part) / parts);
        const uint32_t e = min(e0, b0 + 32 * (uint32_t)(((uint64_t)rounds * (part + 1)) / parts));
        init_tile(c, g, nullptr, tile4, false, lane);
        __syncwarp();
        if (e > b) warp_grid_range<S, false>(c, ch.ent[0], b, e, g.u0, g.v0, tile4, *st, ls, lane, shift);
    }
};

// Tiles with many entries, which k_grid_tiles listed and left unwritten:
// k_grid_heavy, launched as clusters of kHugeCluster CTAs, persistent.  Each
// tile's warps take consecutive shares of its entries, each into its own
// zeroed copy of the tile in shared memory; the copies are then summed cell
// pair by cell pair in a fixed order (onto the plane's current values in an
// accumulating pass) and the tile is written once with coalesced 16-byte
// stores.  Every cell of the plane is written by exactly one CTA: no atomics
// on the planes.
//   1. The huge tiles first, one per cluster (the rank-0 CTA claims the next
//      from a counter; the others read the claim from its shared memory): the
//      cluster's warps share the entries; each CTA sums its warps' copies
//      into its first copy, and after a cluster barrier CTA r sums rows
//      [r T / C, (r + 1) T / C) of the C CTAs' sums, read through distributed
//      shared memory in rank order, and stores them.  Clusters that find no
//      huge tile left go on to
//   2. the other heavy tiles, one per CTA (each CTA claims the next from a
//      counter, which balances tiles of very different weights); the CTA's
//      active warps' copies are summed in warp order.
// Taking the few huge tiles first lets the rest of the launch hide their
// length.
template <int S>
__global__ void __launch_bounds__(256) k_grid_heavy(GridCfg c, ChunkList ch, int k0, int shift, int accumulate,
                                                    float2* __restrict__ planes, HeavyList hl)
{
    extern __shared__ float4 smem4[];
    __shared__ uint32_t s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    HeavyCta<S> m(c, smem4, wid, lane);

    // 1. huge tiles (the count is the same for every CTA: the tiles kernel wrote it)
    const uint32_t nx = min(hl.w[2], hl.cap_x);
    if (nx > 0) {
        const uint32_t rank = cluster_rank();
        const uint32_t claim0 = cluster_map((uint32_t)__cvta_generic_to_shared(&s_item), 0);
        const uint32_t gw = rank * nwarps + wid, ngw = kHugeCluster * nwarps;
        const int rpc = c.T / kHugeCluster;  // tile rows stored per CTA (T >= 16)
        for (;;) {
            if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(hl.w + 3, 1u);
            cluster_sync();
            const uint32_t it = ld_cluster_u32(claim0);
            if (it >= nx) break;  // the same value in every CTA of the cluster
            const TileGeom g = tile_geom(c, k0, (int64_t)hl.w[4 + hl.cap_h + it]);
            float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
            m.grid_share(c, ch, g, __ldg(ch.off[0] + g.tg), __ldg(ch.off[0] + g.tg + 1), gw, ngw, lane, shift);
            __syncthreads();
            for (int i = threadIdx.x; i < (c.T << m.ltp); i += blockDim.x) {
                float4* d0 = smem4 + (i >> m.ltp) * m.p2 + (i & m.pmask);
                float4 a = *d0;
                for (uint32_t q = 1; q < nwarps; ++q) add4(a, d0[q * m.wstride]);
                *d0 = a;
            }
            cluster_sync();
            for (int i = threadIdx.x; i < (rpc << m.ltp); i += blockDim.x) {
                const int row = (int)rank * rpc + (i >> m.ltp), pr = i & m.pmask;
                if (row >= g.wv || 2 * pr >= g.wu) continue;
                float4* dst =
                    reinterpret_cast<float4*>(P0 + (int64_t)plane_row(c, g.v0 + row) * c.n + g.u0 + 2 * pr);
                float4 acc = accumulate ? *dst : make_float4(0.f, 0.f, 0.f, 0.f);
                const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(smem4 + row * m.p2 + pr);
                for (uint32_t q = 0; q < (uint32_t)kHugeCluster; ++q) add4(acc, ld_cluster_f4(cluster_map(a0, q)));
                *dst = acc;
            }
            cluster_sync();  // the copies are read remotely until here
        }
        cluster_sync();  // rank 0's claim is read remotely until here
    }

    // 2. the other heavy tiles
    const uint32_t count = min(hl.w[0], hl.cap_h);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(hl.w + 1, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= count) break;
        const TileGeom g = tile_geom(c, k0, (int64_t)hl.w[4 + it]);
        float2* P0 = planes + (int64_t)g.kl * c.n * c.n;
        const uint32_t b0 = __ldg(ch.off[0] + g.tg), e0 = __ldg(ch.off[0] + g.tg + 1);
        const uint32_t nact = min(nwarps, max(1u, (e0 - b0 + kHeavyPerWarp - 1) / kHeavyPerWarp));
        if ((uint32_t)wid < nact) m.grid_share(c, ch, g, b0, e0, wid, nact, lane, shift);
        __syncthreads();
        // thread i: pair column i mod (T/2) of tile row i / (T/2); a half-warp
        // (T = 32) covers one 256-byte row segment
        for (int i = threadIdx.x; i < (c.T << m.ltp); i += blockDim.x) {
            const int row = i >> m.ltp, pr = i & m.pmask;
            if (row >= g.wv || 2 * pr >= g.wu) continue;
            float4* dst = reinterpret_cast<float4*>(P0 + (int64_t)plane_row(c, g.v0 + row) * c.n + g.u0 + 2 * pr);
            float4 acc = accumulate ? *dst : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4* src = smem4 + row * m.p2 + pr;
            for (uint32_t q = 0; q < nact; ++q, src += m.wstride) add4(acc, *src);
            *dst = acc;
        }
        __syncthreads();  // the next tile's init overwrites the copies, the next claim s_item
    }
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The launch configuration of k_grid_heavy: clusters of kHugeCluster CTAs of
// hw warps (grid: nclusters clusters).
inline cudaLaunchConfig_t heavy_config(cudaLaunchAttribute* at, int hw, size_t smem, int nclusters, cudaStream_t s)
{
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kHugeCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(nclusters * kHugeCluster));
    lc.blockDim = dim3((unsigned)(32 * hw));
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    lc.attrs = at;
    lc.numAttrs = 1;
    return lc;
}

// What launch_grid_s<S> sets and queries once per device (and tile side):
// the shared-memory opt-ins of its two kernels, at the largest size any tile
// side launches them with (the opt-in is a per-kernel ceiling: lowering it for
// one tile side would fail the launches of another), and the co-resident
// k_grid_heavy clusters.  (Two threads that launch first at the same time both
// query; the values are the same.)
struct GridLaunchInfo {
    int clusters;
};

template <int S>
cudaError_t grid_launch_info(int T, size_t tile_bytes, int hw, GridLaunchInfo& out)
{
    static GridLaunchInfo cache[64][7];
    static std::atomic<int> ready[64][7];
    static std::atomic<int> opted[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int lt = 0;
    while ((1 << lt) < T && lt < 6) ++lt;
    const bool cached = dev >= 0 && dev < 64;
    if (cached && ready[dev][lt].load(std::memory_order_acquire)) {
        out = cache[dev][lt];
        return cudaSuccess;
    }
    if (!cached || !opted[dev].load(std::memory_order_acquire)) {
        size_t light_max = 0, heavy_max = 0;
        for (int t = 16; t <= 64; t *= 2) {
            light_max = std::max(light_max, warp_smem_bytes<S>(t) * light_warps(t));
            heavy_max = std::max(heavy_max, warp_smem_bytes<S>(t) * heavy_warps<S>(t));
        }
        if ((e = allow_smem(k_grid_tiles<S>, light_max)) != cudaSuccess) return e;
        if ((e = allow_smem(k_grid_heavy<S>, heavy_max)) != cudaSuccess) return e;
        if (cached) opted[dev].store(1, std::memory_order_release);
    }
    const size_t heavy_bytes = tile_bytes * hw;
    GridLaunchInfo g{0};
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t lc = heavy_config(at, hw, heavy_bytes, sm_count_grid(), nullptr);
    if ((e = cudaOccupancyMaxActiveClusters(&g.clusters, k_grid_heavy<S>, &lc)) != cudaSuccess) return e;
    if (g.clusters < 1) return cudaErrorInvalidConfiguration;
    if (cached) {
        cache[dev][lt] = g;
        ready[dev][lt].store(1, std::memory_order_release);
    }
    out = g;
    return cudaSuccess;
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
    // heavy: [count, claim, huge count, huge claim, tiles, huge tiles]; a
    // ninth of the slots for huge tiles (more than kHugePerWarp >= 512
    // entries each, so at most an eighth as many as heavy ones, which hold
    // more than 64)
    const size_t slots = heavy_words - 4;
    const size_t sx = slots / 9, sh = slots - sx;
    const int hw = heavy_warps<S>(c.T);
    const HeavyList hl{heavy, (uint32_t)(sh < 0x7fffffffu ? sh : 0x7fffffffu),
                       (uint32_t)(sx < 0x7fffffffu ? sx : 0x7fffffffu), (uint32_t)hw * kHugePerWarp};
    const size_t heavy_bytes = tile_bytes * hw;
    GridLaunchInfo info;
    cudaError_t e = grid_launch_info<S>(c.T, tile_bytes, hw, info);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(heavy, 0, 4 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    const unsigned tile_blocks = (unsigned)((nblocks + kTilesPerWarp - 1) / kTilesPerWarp);
    k_grid_tiles<S><<<tile_blocks, 32 * wl, tile_bytes * wl, s>>>(c, ch, k0, ntl, shift ? 1 : 0, accumulate ? 1 : 0,
                                                                  planes, hl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // persistent: as many clusters as are co-resident
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t lc = heavy_config(at, hw, heavy_bytes, info.clusters, s);
    e = cudaLaunchKernelEx(&lc, k_grid_heavy<S>, c, ch, k0, shift ? 1 : 0, accumulate ? 1 : 0, planes, hl);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // reported here; not left for the next launch check to find
        return e;
    }
    return cudaGetLastError();
}

}  // namespace

// A heavy tile holds more than h >= kHeavyMin = 64 entries and a huge one
// more than kHugePerWarp >= 512, so a pass over E entries lists fewer than
// E / 64 and E / 512 of them: four header words and 9 (E / 512 + 1) slots, a
// ninth of them for huge tiles, hold both.
size_t heavy_words_for(int64_t max_entries)
{
    static_assert(kHeavyMin * 8 <= kHugePerWarp, "the list split assumes huge tiles hold 8x the heavy minimum");
    return 4 + 9 * ((size_t)(max_entries > 0 ? max_entries : 0) / (8 * kHeavyMin) + 1);
}

cudaError_t launch_grid(const GridCfg& c, const ChunkList& ch, int k0, int nk, bool shift_sign,
                        bool accumulate, uint32_t* heavy, size_t heavy_words, float2* planes, cudaStream_t s)
{
    if (!heavy || heavy_words < 4) return cudaErrorInvalidValue;
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
