// rick_internal.cuh -- device-side configuration, placement and kernel
// launchers shared by the translation units of librick (GPU side only).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "../../include/rick.h"

namespace rick {

constexpr int kMaxSupport = 16;
constexpr int kPolyTerms = 11;            // degree-10 polynomial per kernel tap
constexpr int kMaxChunksPerPass = 16;
constexpr int kScanBlock = 1024;          // threads of the scan kernels
constexpr int kScanItems = 4;             // items per scan thread
constexpr int kScanTile = kScanBlock * kScanItems;

// Words between consecutive per-tile counters of the counting sort.  With
// few tiles (a small grid), or with a dense uv centre whose few tiles take
// most of the measurements, the busy counters would share a handful of L2
// lines, and the measurements' atomic adds would queue at the same few L2
// slices; spreading the counters up to one 128-byte line each, while they
// take at most max_words words in all, lets every slice take a share.  Large
// grids keep them packed.  Measured on a dense 2048^2 x 16-plane channel of
// 2e7 measurements (65 536 tiles, up to 4e4 entries in one): the sort took
// 1.36 ms with the counters packed (a 2^16-word cap) and 0.81 ms with one
// line each (2^22).  The allocation-free entry point keeps the 2^16-word cap
// (kStaticCounterWords) so that its fixed scratch holds what it documents.
constexpr int64_t kCounterWords = (int64_t)1 << 22;
constexpr int64_t kStaticCounterWords = (int64_t)1 << 16;

__host__ __device__ inline int counter_stride(int64_t ntiles, int64_t max_words = kCounterWords)
{
    int s = 1;
    while (s < 32 && ntiles * s * 2 <= max_words) s *= 2;
    return s;
}

// Everything a kernel needs to place a measurement, by value.
struct GridCfg {
    int n, nw, S, T, log2T, ntu;     // nw: planes in total (channels x planes per channel)
                                     // ntu: tiles per side = ceil(n / T)
    int64_t ntp;                     // tiles per plane = ntu * ntu
    int ntu_log2;                    // log2(ntu) when ntu is a power of two, else -1
    int cstride;                     // words between the per-tile counters (counter_stride)
    float uvscale;                   // cells per wavelength, binary32
    float half_n, half_s;            // n/2, S/2
    float wmin, invdw;               // binary32 plane decision constants
    float lim;                       // n - S - 1: largest first cell - 1
    int kernel;                      // RICK_KERNEL_*
    int uniform;                     // uniform weighting on
    // w-support (Eq. 3's kernel in w): Sw planes per measurement; 1 = nearest
    int Sw;
    float half_sw, wkp, two_over_sw; // Sw/2; Gaussian 1/(2 sigma_w^2) or KB beta_w; 2/Sw
    int fold;                        // RICK_HERMITIAN_FOLD: mirror measurements with w < 0
    // blocks per SM of the sort kernels (measurements per block = M / (SMs x
    // this); 0 = 8), one of the batched autotuner's knobs
    int prep_bpsm;
    // planes this handle grids and transforms: [plane_lo, plane_hi) of the nw
    // (rick_set_plane_range; all by default).  Measurements on other planes
    // are placed, weighted and counted but list no entries.
    int plane_lo, plane_hi;
    // row order of the planes in memory: 0 = natural (row v at v); r > 0 =
    // b-major storage of the split transform, n = 16 N1 with N1 = 2^r: row
    // v = 16 a + b lives at b N1 + a (plane_row), so the rows of each column
    // factor's input (fixed b) are one contiguous run of the plane
    int row_perm;
    // batched imaging: nchan channels with nw_chan w-planes each, channel c
    // owning planes c*nw_chan .. (c+1)*nw_chan-1 and measurements
    // chan_off[c] .. chan_off[c+1]-1; chan_w[c] = (w_min, 1/dw) in binary32.
    int nchan, nw_chan;
    const float2* chan_w;
    const int64_t* chan_off;
    // tap t of a measurement whose footprint starts at f = floor(p - S/2) + 1
    // is g(t + 1 - S/2 - d), d = frac(p - S/2); as a polynomial in z = 2d - 1:
    // g_t = sum_j coef[t][j] z^j (fitted once per handle, see k_fit_taps)
    float coef[kMaxSupport][kPolyTerms];
    // sum_t g_t = sum_j sumc[j] z^j: the tap sum of one axis (set_tap_sum)
    float sumc[kPolyTerms];
};

// Memory row of grid row v of a plane (see GridCfg::row_perm).
__host__ __device__ __forceinline__ int plane_row(const GridCfg& c, int v)
{
    return c.row_perm ? ((v & 15) << c.row_perm) | (v >> 4) : v;
}

// Placement of one measurement: plane, first footprint cell, continuous
// cell coordinates.  Every float->int decision is binary32 with the
// operation order written out (explicit _rn intrinsics, no contraction).
struct Place {
    int k, fu, fv;  // k: the plane (Sw = 1) or the first plane of the w-footprint (may be off the range)
    float pu, pv;
    float pw;       // continuous plane coordinate, plane k's centre at k (Sw > 1)
    bool conj;      // imaged as the Hermitian mirror: use conj(V)
};

__device__ __forceinline__ bool place(const GridCfg& c, float u, float v, float w, Place& p, int chan = 0)
{
    if (!(isfinite(u) && isfinite(v) && isfinite(w))) return false;
    // binary32 negation is exact: the mirror is placed like any measurement
    p.conj = c.fold && w < 0.0f;
    if (p.conj) {
        u = -u;
        v = -v;
        w = -w;
    }
    float pu = __fmaf_rn(u, c.uvscale, c.half_n);
    float pv = __fmaf_rn(v, c.uvscale, c.half_n);
    float au = floorf(__fsub_rn(pu, c.half_s));
    float av = floorf(__fsub_rn(pv, c.half_s));
    if (!(au >= -1.0f && au <= c.lim && av >= -1.0f && av <= c.lim)) return false;
    p.fu = (int)au + 1;
    p.fv = (int)av + 1;
    if (c.nw_chan == 1) {
        p.k = chan;
    } else {
        float wmin = c.wmin, invdw = c.invdw;
        if (c.nchan > 1) {
            const float2 cw = __ldg(c.chan_w + chan);
            wmin = cw.x;
            invdw = cw.y;
        }
        if (c.Sw == 1) {
            float fk = floorf(__fmul_rn(__fsub_rn(w, wmin), invdw));
            const int k = (fk < 0.0f) ? 0 : ((fk > (float)(c.nw_chan - 1)) ? c.nw_chan - 1 : (int)fk);
            p.k = chan * c.nw_chan + k;
        } else {
            // planes fk .. fk + Sw - 1, fk = floor(pw - Sw/2) + 1 (one channel)
            p.pw = __fsub_rn(__fmul_rn(__fsub_rn(w, wmin), invdw), 0.5f);
            p.k = (int)floorf(__fsub_rn(p.pw, c.half_sw)) + 1;
        }
    }
    p.pu = pu;
    p.pv = pv;
    return true;
}

// First footprint cell from a stored continuous coordinate (same rounding
// as place()).
__device__ __forceinline__ int first_cell(const GridCfg& c, float p)
{
    return (int)floorf(__fsub_rn(p, c.half_s)) + 1;
}

// Nearest cell for the density grid.
__device__ __forceinline__ int nearest_cell(const GridCfg& c, float p)
{
    int j = (int)floorf(__fadd_rn(p, 0.5f));
    return j > c.n - 1 ? c.n - 1 : j;
}

// The S (un-normalised) taps of a measurement at continuous coordinate p
// whose first footprint cell is f: Horner evaluation of the fitted
// polynomials; the coefficients are uniform across threads (kernel
// parameters, constant-bank broadcast).
template <int S>
__device__ __forceinline__ void eval_taps(const GridCfg& c, float p, int f, float (&g)[S])
{
    const float d = __fsub_rn(__fsub_rn(p, c.half_s), (float)(f - 1));  // in [0, 1)
    const float z = __fmaf_rn(2.0f, d, -1.0f);
#pragma unroll
    for (int t = 0; t < S; ++t) {
        float a = c.coef[t][kPolyTerms - 1];
#pragma unroll
        for (int j = kPolyTerms - 2; j >= 0; --j) a = __fmaf_rn(a, z, c.coef[t][j]);
        g[t] = a;
    }
}

// Sum of the S taps of one axis: one Horner evaluation of the sum of the tap
// polynomials (normalised taps then sum to 1 to a few binary32 roundings).
__device__ __forceinline__ float tap_sum(const GridCfg& c, float p, int f)
{
    const float d = __fsub_rn(__fsub_rn(p, c.half_s), (float)(f - 1));
    const float z = __fmaf_rn(2.0f, d, -1.0f);
    float s = c.sumc[kPolyTerms - 1];
#pragma unroll
    for (int j = kPolyTerms - 2; j >= 0; --j) s = __fmaf_rn(s, z, c.sumc[j]);
    return s;
}

constexpr int kMaxWSupport = 16;

// Un-normalised kernel in w at x plane widths from the measurement (Sw > 1).
__device__ __forceinline__ float w_kernel(const GridCfg& c, float x)
{
    if (c.kernel == RICK_KERNEL_GAUSS) return __expf(-x * x * c.wkp);
    const float z = x * c.two_over_sw;
    return cyl_bessel_i0f(c.wkp * sqrtf(fmaxf(0.0f, 1.0f - z * z)));
}

// 1 / (sum of a placed measurement's Sw w-taps); its weight on plane p.k + t
// is w_kernel(c, (p.k + t) - p.pw) times this.
__device__ __forceinline__ float w_tap_norm(const GridCfg& c, const Place& p)
{
    float s = 0.0f;
    for (int t = 0; t < c.Sw; ++t) s += w_kernel(c, __fsub_rn((float)(p.k + t), p.pw));
    return 1.0f / s;
}

// Coefficients of the tap-sum polynomial from the S tap polynomials (host).
inline void set_tap_sum(GridCfg& c)
{
    for (int j = 0; j < kPolyTerms; ++j) {
        double s = 0.0;
        for (int t = 0; t < c.S; ++t) s += (double)c.coef[t][j];
        c.sumc[j] = (float)s;
    }
}

// Whether a measurement with finite placement also has a finite weight and value.
__device__ __forceinline__ bool finite_value(float wt, float2 vis)
{
    return isfinite(wt) && isfinite(vis.x) && isfinite(vis.y);
}

// One gridding pass: up to kMaxChunksPerPass sorted chunks.
struct ChunkList {
    const uint32_t* off[kMaxChunksPerPass];  // [ntiles + 1] start offsets
    const float4* ent[kMaxChunksPerPass];    // (pu, pv, re, im) entries, re/im already
                                             // multiplied by weight / (sum of u taps * sum of v taps)
    int count;
};

// Device-resident counters of a handle.
struct Counters {
    unsigned long long gridded, dropped, entries;
    unsigned long long err;          // a bounded wait ran out: bit 0 k_colstack, 1 k_colfft
    double sum_w;
};

// ---------------------------------------------------------------- launchers
cudaError_t launch_density(const GridCfg& c, const float* u, const float* v, const float* w,
                           const float* wt, const float2* vis, int64_t m, uint32_t* density,
                           cudaStream_t s);
cudaError_t launch_count(const GridCfg& c, const float* u, const float* v, const float* w,
                         const float* wt, const float2* vis, int64_t m, uint32_t* counts,
                         cudaStream_t s);
// counts[i * stride] for i < len -> offsets[0..len] (packed, exclusive, total
// last) and cursor[i * stride] = offsets[i]; counts may alias cursor
cudaError_t launch_scan(const uint32_t* counts, int64_t len, int stride, uint32_t* offsets, uint32_t* cursor,
                        uint32_t* block_sums, cudaStream_t s);
// chan_sw: per-channel weight sums (NULL: ctr->sum_w, single channel)
cudaError_t launch_scatter(const GridCfg& c, const float* u, const float* v, const float* w,
                           const float* wt, const float2* vis, int64_t m, const uint32_t* density,
                           uint32_t* cursor, float4* entries, Counters* ctr, double* chan_sw, cudaStream_t s);
// heavy: scratch of heavy_words >= 4 words for the lists of heavily populated
// tiles (four counters, then one word per tile; a tile that does not fit is
// gridded by one warp, correct but slower).  heavy_words_for() gives the size
// that never overflows for a pass over at most max_entries entries.
cudaError_t launch_grid(const GridCfg& c, const ChunkList& chunks, int k0, int nk, bool shift_sign,
                        bool accumulate, uint32_t* heavy, size_t heavy_words, float2* planes, cudaStream_t s);
size_t heavy_words_for(int64_t max_entries);
cudaError_t launch_taper(const GridCfg& c, double kernel_param, float* taper, cudaStream_t s);
// The Fourier transform of the w-kernel at xi_j = xi_max j / (len - 1), j < len.
cudaError_t launch_wcorr(const GridCfg& c, double xi_max, int len, float* out, cudaStream_t s);
// Fit the tap polynomials (coef: float[S][kPolyTerms]) and report the largest
// binary32 evaluation error relative to the kernel's peak in *max_err.
cudaError_t launch_fit_taps(const GridCfg& c, double kernel_param, float* coef, double* max_err, cudaStream_t s);

constexpr int kWcorrLen = 4096;  // samples of the grid correction in w
constexpr float kMinWcorr = 1e-2f;  // smallest grid correction in w accepted over the image

struct StackArgs {
    int n, k0, nk;
    const float* wcorr;              // grid correction in w (w-support > 1), else NULL:
    float wc_scale;                  // table index per unit of -(n - 1)
    float dl2_hi, dl2_lo;            // pixel_rad^2 as a float pair
    float wb_hi, wb_lo;              // w_min + dw/2 as a float pair
    float dw_hi, dw_lo;              // dw as a float pair
    int first, last;                 // first / last plane group
    unsigned flags;
    // k_colstack's bounded waits: the limit of one wait in ns (0: 1 s), and
    // a test hook: 1 + the pipeline slot whose copy the producer leaves out
    // (0: none), so that every wait on it runs out and the error path runs
    unsigned long long wait_ns;
    int skip_slot1;
    // k_colstack: the group's first plane in the plane buffer (a channel of a
    // batch), 0 for single images
    int plane0;
    // k_colstack over several channels of a batch in one launch (blockIdx.z
    // = channel chan0 + z, nk planes each from plane0 + z nk): per channel
    // (w_min + dw/2, dw) as float pairs {wb_hi, wb_lo, dw_hi, dw_lo}; the
    // weight sums and images of consecutive channels follow one another
    // (img_stride floats apart).  NULL: one image.
    const float4* chan_screen;
    int chan0;
    long long img_stride;
};
// The grid correction in w at a pixel with n - 1 = nm1 (linear interpolation
// of the table; 1 without w-support).
__device__ __forceinline__ float wcorr_at(const StackArgs& a, float nm1)
{
    if (!a.wcorr) return 1.0f;
    const float x = fminf(-nm1 * a.wc_scale, (float)(kWcorrLen - 1));
    const int j = min((int)x, kWcorrLen - 2);
    const float f = x - (float)j;
    const float c0 = __ldg(a.wcorr + j), c1 = __ldg(a.wcorr + j + 1);
    return __fmaf_rn(f, c1 - c0, c0);
}

// sum_w: the weight sum the image is normalised by (device)
// n = n1 * n2 split of the column transform for k_colstack (power-of-two n in
// [64, 16384]: n2 = 16, n1 = n / 16); false: use cuFFT 2D + k_stack
bool colstack_shape(int n, int* n1, int* n2);
// screen + stack of a group whose rows and first column factor are transformed
// (cuFFT), the last column factor done here; err: Counters::err
// map: a CUtensorMap (128 bytes, 64-byte aligned) from encode_colstack_map
// for the plane buffer the group is in
cudaError_t encode_colstack_map(void* map, const float2* planes, int n, int planes_in_buffer);
// nchan > 1: the channels a.chan0 .. a.chan0 + nchan - 1 of a batch in one
// launch (a.chan_screen set; sum_w and image are the first channel's)
cudaError_t launch_colstack(const void* map, const StackArgs& a, int n1, int n2, float2* acc, const float* taper,
                            const double* sum_w, void* image, unsigned long long* err, cudaStream_t s,
                            int nchan = 1);
// adjoint of launch_colstack: planes of the group from the image gradient
// (rows 16 f1 + b after the last column factor's adjoint); cuFFT's forward
// first column factor and rows complete the forward 2D transform
// the first column factor of the split transform for a group of nk planes
// (k_colfft, rick_colfft.cu): rows 16 a + b -> rows 16 f1 + b in place, the
// N1 = n / 16-point DFT with exponent sign (+1 imaging, -1 adjoint); map
// from encode_colfft_map for the plane buffer, tw = exp(+2 pi i j / N1)
cudaError_t encode_colfft_map(void* map, const float2* planes, int n, int planes_in_buffer);
cudaError_t launch_colfft(const void* map, const float2* tw, float2* planes, int n, int nk, int sign,
                          unsigned long long wait_ns, unsigned long long* err, cudaStream_t s);
cudaError_t launch_spreadcol(const StackArgs& a, int n1, int n2, const void* rimg, const float* taper,
                             const double* sum_w, float2* planes, cudaStream_t s);
cudaError_t launch_stack(const StackArgs& a, const float2* planes, float2* acc, const float* taper,
                         const double* sum_w, void* image, cudaStream_t s);

cudaError_t launch_spread(const StackArgs& a, const void* rimg, const float* taper, const double* sum_w,
                          float2* planes, cudaStream_t s);
// adjoint: sort measurements by the tile of their first footprint cell
// (no duplication), then gather each measurement's footprint of a plane group
cudaError_t launch_primary_count(const GridCfg& c, const float* u, const float* v, const float* w,
                                 const float* wt, int64_t m, uint32_t* counts, cudaStream_t s);
cudaError_t launch_primary_scatter(const GridCfg& c, const float* u, const float* v, const float* w,
                                   const float* wt, int64_t m, uint32_t* cursor, uint32_t* perm,
                                   cudaStream_t s);
cudaError_t launch_degrid_gather(const GridCfg& c, const uint32_t* perm, const uint32_t* offsets, int k0, int nk,
                                 const float2* planes, const float* u, const float* v, const float* w,
                                 const float* wt, const uint32_t* density, float2* grad, cudaStream_t s);

size_t scan_block_sums_len(int64_t len);

// Parameter checks of rick_create (fills the derived configuration).
rick_status validate_params(const rick_params* p, GridCfg* c, double* kparam, char* msg, size_t msglen);

}  // namespace rick

namespace rick {
enum Phase { kPhasePrep = 0, kPhaseGrid, kPhaseFft, kPhaseStack, kPhaseDegrid, kPhaseColfft, kNumPhases };

// CUDA-event timer per phase: events are recorded on the stream and only
// resolved (elapsed time summed) when the caller asks for the totals.
struct PhaseTimer {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[kNumPhases];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
    double ms[kNumPhases] = {};
    int64_t calls[kNumPhases] = {};
    int64_t launches = 0;
    cudaEvent_t open_start[kNumPhases] = {};
};
}  // namespace rick

// The handle.
struct rick_imager {
    rick_params p;
    rick::GridCfg cfg;
    double kernel_param;             // resolved sigma / beta
    int device;
    cudaStream_t stream;
    int G;                           // planes per group
    // device buffers
    float* taper;                    // [n]
    float2* planes;                  // [G][n][n]
    float2* acc;                     // [n][n] image accumulator (several groups)
    uint32_t* cursor;                // [ntiles] counts / scatter cursors
    uint32_t* block_sums;            // scan block totals
    uint32_t* density;               // [n][n] uniform weighting counts
    rick::Counters* ctr;             // device counters
    double* one;                     // device 1.0: the weight sum of unweighted prediction
    float* wcorr;                    // [kWcorrLen] grid correction in w (w-support > 1)
    float wc_scale;
    void* fft_work;
    size_t fft_work_bytes;
    std::map<int, cufftHandle> plans;// (kind, batch) -> plan
    alignas(64) unsigned char colmap[128];  // tensor map of `planes` for k_colstack
    bool colmap_ready;
    alignas(64) unsigned char cfmap[128];   // tensor map of `planes` for k_colfft
    bool cfmap_ready;
    // batched imaging with the split transform: the same maps for `planes2`
    bool batch_split;
    alignas(64) unsigned char colmap2[128];
    alignas(64) unsigned char cfmap2[128];
    float2* cf_tw;                   // [n / 16] exp(+2 pi i j / (n / 16)) for k_colfft
    struct Chunk {
        uint32_t* off;
        float4* ent;
        int64_t cap;
    };
    std::vector<Chunk> chunks;
    cudaMemPool_t pool;              // stream-ordered pool for chunk buffers
    bool density_frozen;
    bool user_density;               // density filled by rick_add_density
    // host staging for rick_image_host
    float* stage;
    size_t stage_bytes;
    float* img_dev;
    size_t img_bytes;
    // pipelined host path (rick_image_host_async): two slots of device
    // inputs and images; uploads and downloads on their own streams, ordered
    // against the compute stream by events
    bool async_ready;
    cudaStream_t h2d, d2h;
    float* astage[2];
    float* aimg[2];
    size_t astage_bytes, aimg_bytes;
    cudaEvent_t ev_staged[2], ev_computed[2], ev_fetched[2];
    int aslot;
    size_t bytes_held;
    rick::PhaseTimer timer;
    // batched imaging (rick_create_batch): per-channel w-ranges and sums,
    // persistent entry buffers, and the captured graph of one batch step
    bool batch;
    int nchan;
    std::vector<double> chan_wmin, chan_wmax;
    float2* chan_w;                  // device [nchan] (w_min, 1/dw) binary32
    int64_t* chan_off;               // device [nchan + 1]
    double* chan_sw;                 // device [nchan] weight sums
    float4* chan_scr;                // device [nchan] w-screen constants (StackArgs::chan_screen)
    std::vector<int64_t> chan_off_host;
    uint32_t* b_off;                 // device [ntiles + 1]
    float4* b_ent;                   // device entries
    int64_t b_cap;
    uint32_t* b_heavy;               // gridder's heavy-tile list for b_cap entries
    size_t b_heavy_words;
    // pipelined plane groups (batched, two or more groups): a second plane
    // buffer; group g is gridded on the handle's stream into buffer g % 2 while
    // group g - 1 is transformed and stacked on fft_stream
    float2* planes2;
    cudaStream_t fft_stream;
    cudaEvent_t ev_fork, ev_gridded[2], ev_free[2];
    cudaGraphExec_t graph;
    const void* graph_key[7];
    int64_t graph_m;
    // normalisation weight sum supplied by the caller (rick_set_weight_sum):
    // used instead of the handle's own sum when sw_given
    bool sw_given;
    double sw_host;
    double* sw_dev;
    // test hook of k_colstack's bounded waits (rick_debug_colstack)
    int dbg_skip_slot1;
    unsigned long long dbg_wait_ns;
    char last_error[512];
};
