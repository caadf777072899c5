// rick_api.cu -- the C ABI of librick (include/rick.h): handle, parameter
// checks, device memory plan, cuFFT plans and the step sequence of the
// workflow in Sec. 2.1 (grid -> per-plane FFT -> w-correction + reduction).
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "rick_internal.cuh"

using namespace rick;

namespace {

rick_status fail(rick_handle h, rick_status s, const char* fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->last_error, sizeof(h->last_error), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define RICK_CU(h, expr)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(h, RICK_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

#define RICK_FFT(h, expr)                                                           \
    do {                                                                            \
        cufftResult r_ = (expr);                                                    \
        if (r_ != CUFFT_SUCCESS) return fail(h, RICK_ERR_CUFFT, "%s: cufft error %d", #expr, (int)r_); \
    } while (0)

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int ilog2(int x)
{
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

// Parameter checks; on success fills the derived configuration.
rick_status check_params(const rick_params* p, GridCfg* c, double* kparam, char* msg, size_t msglen)
{
    if (!p) {
        snprintf(msg, msglen, "params is NULL");
        return RICK_ERR_ARG;
    }
    if (p->n < 4 || (p->n & 1) || p->n > 32768) {
        snprintf(msg, msglen, "n must be even and in [4, 32768] (got %d)", p->n);
        return RICK_ERR_ARG;
    }
    if (p->nw < 1 || p->nw > 65535) {
        snprintf(msg, msglen, "nw must be in [1, 65535] (got %d)", p->nw);
        return RICK_ERR_ARG;
    }
    if (!(p->pixel_rad > 0.0) || !std::isfinite(p->pixel_rad)) {
        snprintf(msg, msglen, "pixel_rad must be positive and finite");
        return RICK_ERR_ARG;
    }
    if (!std::isfinite(p->w_min) || !std::isfinite(p->w_max) ||
        (p->nw > 1 && !(p->w_max > p->w_min)) || (p->nw == 1 && p->w_max < p->w_min)) {
        snprintf(msg, msglen, "need finite w_min < w_max (w_min <= w_max when nw == 1)");
        return RICK_ERR_ARG;
    }
    if (p->kernel != RICK_KERNEL_GAUSS && p->kernel != RICK_KERNEL_KB) {
        snprintf(msg, msglen, "unknown kernel %d", p->kernel);
        return RICK_ERR_ARG;
    }
    if (p->support < 1 || p->support > kMaxSupport || 2 * p->support > p->n) {
        snprintf(msg, msglen, "support must be in [1, %d] and at most n/2 (got %d)", kMaxSupport, p->support);
        return RICK_ERR_ARG;
    }
    if (!(p->kernel_param >= 0.0) || !std::isfinite(p->kernel_param)) {
        snprintf(msg, msglen, "kernel_param must be >= 0 and finite");
        return RICK_ERR_ARG;
    }
    if (p->plane_group < 0) {
        snprintf(msg, msglen, "plane_group must be >= 0");
        return RICK_ERR_ARG;
    }
    int T = p->tile ? p->tile : 32;
    if (T != 16 && T != 32 && T != 64) {
        snprintf(msg, msglen, "tile must be 0, 16, 32 or 64 (got %d)", p->tile);
        return RICK_ERR_ARG;
    }
    if (T < p->support) {
        if (p->tile) {
            snprintf(msg, msglen, "tile %d smaller than support %d", T, p->support);
            return RICK_ERR_ARG;
        }
        T = 32;
    }
    const uint32_t known = RICK_GRID_CORRECT | RICK_REAL_IMAGE | RICK_APPLY_N | RICK_UNIFORM_WEIGHT |
                           RICK_HERMITIAN_FOLD | RICK_FFT_2D | RICK_FFT_SPLIT;
    if (p->flags & ~known) {
        snprintf(msg, msglen, "unknown flags 0x%x", p->flags & ~known);
        return RICK_ERR_ARG;
    }
    if ((p->flags & RICK_FFT_2D) && (p->flags & RICK_FFT_SPLIT)) {
        snprintf(msg, msglen, "RICK_FFT_2D and RICK_FFT_SPLIT exclude each other");
        return RICK_ERR_ARG;
    }
    {
        int n1 = 0, n2 = 0;
        if ((p->flags & RICK_FFT_SPLIT) && !colstack_shape(p->n, &n1, &n2)) {
            snprintf(msg, msglen, "RICK_FFT_SPLIT needs a power-of-two n in [64, 16384] (got %d)", p->n);
            return RICK_ERR_ARG;
        }
    }
    if ((p->flags & RICK_HERMITIAN_FOLD) && !(p->flags & RICK_REAL_IMAGE)) {
        snprintf(msg, msglen, "RICK_HERMITIAN_FOLD changes the imaginary part: it needs RICK_REAL_IMAGE");
        return RICK_ERR_ARG;
    }
    double kp = p->kernel_param;
    if (kp == 0.0) kp = (p->kernel == RICK_KERNEL_GAUSS) ? p->support / 6.0 : 2.34 * p->support;
    *kparam = kp;
    c->n = p->n;
    c->nw = p->nw;
    c->S = p->support;
    c->T = T;
    c->log2T = ilog2(T);
    c->ntu = (p->n + T - 1) / T;
    c->ntp = (int64_t)c->ntu * c->ntu;
    c->ntu_log2 = (c->ntu & (c->ntu - 1)) == 0 ? ilog2(c->ntu) : -1;
    c->cstride = counter_stride((int64_t)c->nw * c->ntp);
    c->uvscale = (float)((double)p->n * p->pixel_rad);
    c->half_n = (float)(p->n / 2);
    c->half_s = (float)(0.5 * p->support);
    c->wmin = (float)p->w_min;
    const double dw = (p->nw > 1) ? (p->w_max - p->w_min) / p->nw : (p->w_max - p->w_min);
    c->invdw = (p->nw > 1) ? (float)(1.0 / dw) : 0.0f;
    c->lim = (float)(p->n - p->support - 1);
    c->kernel = p->kernel;
    if (p->w_support < 0 || p->w_support > kMaxWSupport || p->w_support > p->nw) {
        snprintf(msg, msglen, "w_support must be in [0, min(16, nw)] (got %d)", p->w_support);
        return RICK_ERR_ARG;
    }
    c->Sw = p->w_support > 1 ? p->w_support : 1;
    c->half_sw = 0.5f * (float)c->Sw;
    c->two_over_sw = 2.0f / (float)c->Sw;
    c->wkp = (p->kernel == RICK_KERNEL_GAUSS) ? (float)(1.0 / (2.0 * (c->Sw / 6.0) * (c->Sw / 6.0)))
                                              : (float)(2.34 * c->Sw);
    c->uniform = (p->flags & RICK_UNIFORM_WEIGHT) ? 1 : 0;
    c->fold = (p->flags & RICK_HERMITIAN_FOLD) ? 1 : 0;
    c->nchan = 1;
    c->nw_chan = p->nw;
    c->chan_w = nullptr;
    c->chan_off = nullptr;
    c->plane_lo = 0;
    c->plane_hi = p->nw;
    c->row_perm = 0;
    (void)is_pow2;
    return RICK_OK;
}

void split(double x, float* hi, float* lo)
{
    *hi = (float)x;
    *lo = (float)(x - (double)*hi);
}

size_t plane_bytes(const rick_params* p) { return (size_t)p->n * p->n * sizeof(float2); }

// Plans of a handle, one per (kind, batch):
//   kPlan2D    2D n x n transforms of `batch` planes
//   kPlanRows  1D n-point transforms of the rows of `batch` planes
// (the first column factor of the split transform is k_colfft's, the last
// k_colstack's or k_spreadcol's)
enum { kPlan2D = 0, kPlanRows = 1 };
// smallest n for the split column transform without RICK_FFT_SPLIT, from
// measured single images (ms, split / cuFFT 2D plan + k_stack): 256^2 x 8
// 0.104 / 0.099, 512^2 x 16 0.189 / 0.175, 1024^2 x 16 0.353 / 0.351,
// 2048^2 x 16 1.169 / 1.278, 4096^2 x 32 5.06 / 6.32 (small planes stay
// partly in L2 through the 2D plan's passes)
constexpr int kSplitMinN = 2048;
// the same for batched imaging, whose groups hold many planes
constexpr int kBatchSplitMinN = 1024;

// The split transform (cuFFT on the rows, k_colfft on the first column
// factor, the last factor fused with the screen) for single images: n >=
// 2048 by default, any eligible n with RICK_FFT_SPLIT, never with RICK_FFT_2D.
bool use_split(const rick_params& p, int* n1, int* n2)
{
    if (!colstack_shape(p.n, n1, n2)) return false;
    if (p.flags & RICK_FFT_SPLIT) return true;
    return !(p.flags & RICK_FFT_2D) && p.n >= kSplitMinN;
}

rick_status get_plan(rick_handle h, int batch, cufftHandle* out, int kind = kPlan2D)
{
    const int key = (kind << 24) | batch;
    auto it = h->plans.find(key);
    if (it != h->plans.end()) {
        *out = it->second;
        return RICK_OK;
    }
    cufftHandle plan;
    RICK_FFT(h, cufftCreate(&plan));
    RICK_FFT(h, cufftSetAutoAllocation(plan, 0));
    const int n = h->p.n;
    size_t work = 0;
    const long long dist = (long long)n * n;
    cufftResult r;
    if (kind == kPlan2D) {
        int dims[2] = {n, n};
        r = cufftMakePlanMany(plan, 2, dims, nullptr, 1, (int)dist, nullptr, 1, (int)dist, CUFFT_C2C, batch, &work);
    } else {
        int dims[1] = {n};
        r = cufftMakePlanMany(plan, 1, dims, nullptr, 1, n, nullptr, 1, n, CUFFT_C2C, batch * n, &work);
    }
    if (r != CUFFT_SUCCESS) {
        cufftDestroy(plan);
        return fail(h, RICK_ERR_CUFFT, "cufftMakePlanMany(kind=%d, n=%d, batch=%d): error %d", kind, n, batch,
                    (int)r);
    }
    if (work > h->fft_work_bytes) {
        size_t fr = 0, tot = 0;
        RICK_CU(h, cudaMemGetInfo(&fr, &tot));
        if (work - h->fft_work_bytes + (64u << 20) > fr) {
            cufftDestroy(plan);
            return fail(h, RICK_ERR_OOM, "cuFFT work area of %zu bytes does not fit", work);
        }
        if (h->fft_work) {
            RICK_CU(h, cudaStreamSynchronize(h->stream));
            cudaFree(h->fft_work);
            h->bytes_held -= h->fft_work_bytes;
            h->fft_work = nullptr;
            h->fft_work_bytes = 0;
        }
        RICK_CU(h, cudaMalloc(&h->fft_work, work));
        h->fft_work_bytes = work;
        h->bytes_held += work;
        for (auto& kv : h->plans) RICK_FFT(h, cufftSetWorkArea(kv.second, h->fft_work));
    }
    RICK_FFT(h, cufftSetWorkArea(plan, h->fft_work));
    RICK_FFT(h, cufftSetStream(plan, h->stream));
    h->plans[key] = plan;
    *out = plan;
    return RICK_OK;
}

void free_chunks(rick_handle h)
{
    for (auto& c : h->chunks) {
        cudaFreeAsync(c.off, h->stream);
        cudaFreeAsync(c.ent, h->stream);
        h->bytes_held -= (size_t)(h->cfg.nw * h->cfg.ntp + 1) * sizeof(uint32_t) + (size_t)c.cap * sizeof(float4);
    }
    h->chunks.clear();
}

// Records CUDA events around one phase when timing is on.
struct PhaseScope {
    rick_handle h;
    Phase ph;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    PhaseScope(rick_handle h_, Phase ph_) : h(h_), ph(ph_)
    {
        if (!h->timer.on) return;
        if (!h->timer.spare.empty()) {
            ev = h->timer.spare.back();
            h->timer.spare.pop_back();
        } else if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
            ev = {nullptr, nullptr};
            return;
        }
        cudaEventRecord(ev.first, h->stream);
    }
    ~PhaseScope()
    {
        if (!ev.first) return;
        cudaEventRecord(ev.second, h->stream);
        h->timer.pending[ph].push_back(ev);
    }
};

void count_launches(rick_handle h, int64_t n) { h->timer.launches += n; }

void resolve_timer(rick_handle h, bool accumulate)
{
    for (int ph = 0; ph < kNumPhases; ++ph) {
        for (auto& ev : h->timer.pending[ph]) {
            float ms = 0.f;
            if (accumulate && cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
                h->timer.ms[ph] += ms;
                h->timer.calls[ph] += 1;
            }
            h->timer.spare.push_back(ev);
        }
        h->timer.pending[ph].clear();
    }
}

int64_t entries_bound(const GridCfg& c, int64_t nvis) { return nvis * (c.S > 1 ? 4 : 1) * c.Sw; }

rick_status check_vis_args(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                           int64_t nvis)
{
    if (nvis < 0) return fail(h, RICK_ERR_ARG, "nvis must be >= 0 (got %lld)", (long long)nvis);
    if (nvis > 0 && (!vis || !u || !v || !w)) return fail(h, RICK_ERR_ARG, "vis, u, v, w must not be NULL");
    if (nvis > (int64_t)1 << 30) return fail(h, RICK_ERR_ARG, "at most 2^30 measurements per call");
    return RICK_OK;
}

// The weight sum images are normalised by: the caller's (rick_set_weight_sum)
// or the handle's own (device).
const double* norm_sum(rick_handle h) { return h->sw_given ? h->sw_dev : &h->ctr->sum_w; }

// The twiddle table and tensor map of k_colfft (the first column factor of
// the split transform), made on first use: exp(+2 pi i j / N1), j < N1, in
// FP64 rounded once to binary32.
rick_status colfft_ready(rick_handle h)
{
    if (h->cfmap_ready) return RICK_OK;
    const int n1 = h->p.n / 16;
    std::vector<float2> tw(n1);
    for (int j = 0; j < n1; ++j) {
        const double a = 6.283185307179586476925 * (double)j / (double)n1;
        tw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    if (!h->cf_tw) {
        RICK_CU(h, cudaMalloc((void**)&h->cf_tw, sizeof(float2) * n1));
        h->bytes_held += sizeof(float2) * n1;
    }
    RICK_CU(h, cudaMemcpy(h->cf_tw, tw.data(), sizeof(float2) * n1, cudaMemcpyHostToDevice));
    RICK_CU(h, encode_colfft_map(h->cfmap, h->planes, h->p.n, h->G));
    h->cfmap_ready = true;
    return RICK_OK;
}

// Grid planes [k0, k0 + nk) of every stored chunk into `planes`: the
// handle's own buffer (its row order) or a caller's (natural rows).
rick_status grid_pass(rick_handle h, int k0, int nk, bool shift, float2* planes, bool natural_rows = false)
{
    PhaseScope scope(h, kPhaseGrid);
    GridCfg cfg = h->cfg;
    if (natural_rows) cfg.row_perm = 0;
    const size_t nch = h->chunks.size();
    size_t c0 = 0;
    do {
        ChunkList cl{};
        cl.count = 0;
        for (size_t q = c0; q < nch && cl.count < kMaxChunksPerPass; ++q, ++cl.count) {
            cl.off[cl.count] = h->chunks[q].off;
            cl.ent[cl.count] = h->chunks[q].ent;
        }
        // the heavy-tile list (used when the pass has one chunk) is sized
        // for that chunk's entry bound, stream-ordered from the pool
        const size_t words = cl.count == 1 ? heavy_words_for(h->chunks[c0].cap) : 4;
        uint32_t* heavy = nullptr;
        RICK_CU(h, cudaMallocFromPoolAsync((void**)&heavy, words * sizeof(uint32_t), h->pool, h->stream));
        const cudaError_t e = launch_grid(cfg, cl, k0, nk, shift, c0 > 0, heavy, words, planes, h->stream);
        cudaFreeAsync(heavy, h->stream);
        RICK_CU(h, e);
        count_launches(h, 2);
        c0 += kMaxChunksPerPass;
    } while (c0 < nch);
    return RICK_OK;
}

}  // namespace

namespace rick {
rick_status validate_params(const rick_params* p, GridCfg* c, double* kparam, char* msg, size_t msglen)
{
    return check_params(p, c, kparam, msg, msglen);
}
}  // namespace rick

extern "C" {

rick_status rick_params_default(rick_params* p)
{
    if (!p) return RICK_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->n = 256;
    p->nw = 8;
    p->pixel_rad = 1.3635e-4;
    p->w_min = -50.0;
    p->w_max = 50.0;
    p->kernel = RICK_KERNEL_GAUSS;
    p->support = 7;
    p->flags = RICK_GRID_CORRECT | RICK_REAL_IMAGE;
    return RICK_OK;
}

const char* rick_status_string(rick_status s)
{
    switch (s) {
        case RICK_OK: return "RICK_OK";
        case RICK_ERR_ARG: return "RICK_ERR_ARG";
        case RICK_ERR_OOM: return "RICK_ERR_OOM";
        case RICK_ERR_CUDA: return "RICK_ERR_CUDA";
        case RICK_ERR_CUFFT: return "RICK_ERR_CUFFT";
        case RICK_ERR_TIMEOUT: return "RICK_ERR_TIMEOUT";
        case RICK_ERR_STATE: return "RICK_ERR_STATE";
        default: return "RICK_ERR_UNKNOWN";
    }
}

// The message of the last rick_create / rick_create_batch that failed on
// this thread (the handle it was building is gone).
static thread_local char g_create_error[512];

const char* rick_last_error(rick_handle h)
{
    if (h) return h->last_error;
    return g_create_error[0] ? g_create_error : "null handle";
}

rick_status rick_workspace_size(const rick_params* p, int64_t max_vis, size_t* bytes)
{
    GridCfg c;
    double kp;
    char msg[256];
    if (!bytes || max_vis < 0) return RICK_ERR_ARG;
    rick_status s = check_params(p, &c, &kp, msg, sizeof(msg));
    if (s) return s;
    const int G = p->plane_group ? (p->plane_group < p->nw ? p->plane_group : p->nw) : p->nw;
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    size_t b = (size_t)G * plane_bytes(p);                           // planes
    if (G < p->nw) b += plane_bytes(p);                              // image accumulator
    b += (size_t)c.n * sizeof(float);                                // taper
    b += (size_t)ntiles * c.cstride * sizeof(uint32_t) + sizeof(uint32_t);  // padded counters / cursor
    b += (size_t)(ntiles + 1) * sizeof(uint32_t);                          // offsets
    b += scan_block_sums_len(ntiles) * sizeof(uint32_t);
    b += (size_t)entries_bound(c, max_vis) * sizeof(float4);         // entries
    b += heavy_words_for(entries_bound(c, max_vis)) * sizeof(uint32_t);  // gridder's heavy-tile list
    if (p->flags & RICK_UNIFORM_WEIGHT) b += (size_t)c.n * c.n * sizeof(uint32_t);
    b += plane_bytes(p);                                             // cuFFT work area (estimate)
    *bytes = b;
    return RICK_OK;
}

static rick_status create_impl(const rick_params* p, int nchan, const double* w_min, const double* w_max,
                               rick_handle* out)
{
    if (!out) return RICK_ERR_ARG;
    *out = nullptr;
    rick_imager* h = new (std::nothrow) rick_imager();
    if (!h) return RICK_ERR_OOM;
    h->last_error[0] = 0;
    g_create_error[0] = 0;
    rick_status s = check_params(p, &h->cfg, &h->kernel_param, h->last_error, sizeof(h->last_error));
    if (s) {
        // the handle is not returned: its message stays reachable through rick_last_error(NULL)
        snprintf(g_create_error, sizeof(g_create_error), "%s", h->last_error);
        delete h;
        return s;
    }
    if (nchan < 1 || nchan > 65535 || (int64_t)nchan * p->nw > 65535) {
        delete h;
        return RICK_ERR_ARG;
    }
    if (nchan > 1 || w_min) {
        if (!w_min || !w_max || (p->flags & RICK_UNIFORM_WEIGHT) || p->w_support > 1) {
            delete h;
            return RICK_ERR_ARG;
        }
        for (int c = 0; c < nchan; ++c)
            if (!std::isfinite(w_min[c]) || !std::isfinite(w_max[c]) || (p->nw > 1 && !(w_max[c] > w_min[c])) ||
                w_max[c] < w_min[c]) {
                delete h;
                return RICK_ERR_ARG;
            }
        h->batch = true;
        h->cfg.nchan = nchan;
        h->cfg.nw_chan = p->nw;
        h->cfg.nw = nchan * p->nw;
        h->cfg.plane_hi = h->cfg.nw;
        h->cfg.cstride = counter_stride((int64_t)h->cfg.nw * h->cfg.ntp);
        h->nchan = nchan;
        h->chan_wmin.assign(w_min, w_min + nchan);
        h->chan_wmax.assign(w_max, w_max + nchan);
    } else {
        h->nchan = 1;
    }
    h->p = *p;
    h->stream = nullptr;
    cudaGetDevice(&h->device);
    {
        // a private stream-ordered pool that keeps freed chunk memory mapped,
        // so per-call entry buffers cost no remapping
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = h->device;
        if (cudaMemPoolCreate(&h->pool, &props) != cudaSuccess) {
            delete h;
            return RICK_ERR_CUDA;
        }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }

    const GridCfg& c = h->cfg;
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete h;
        return RICK_ERR_CUDA;
    }
    // plane group: as requested, else as many planes as fit in 60 % of free memory;
    // in batched imaging a group holds whole channels
    const size_t pb = plane_bytes(p);
    const int NW = c.nw;
    int G = p->plane_group ? p->plane_group : NW;
    if (G > NW) G = NW;
    if (!p->plane_group) {
        // planes + cuFFT's work area: the 2D plan may need as much as the
        // planes, the split transform's row plan far less
        int n1 = 0, n2 = 0;
        const bool split = !h->batch && use_split(*p, &n1, &n2);
        const size_t fit = split ? (size_t)(0.7 * (double)fr) / (pb ? pb : 1)
                                 : (size_t)(0.6 * (double)fr) / (pb ? 2 * pb : 1);
        if ((size_t)G > fit) G = (int)(fit > 0 ? fit : 1);
        // groups of equal size (no short last group)
        const int ngroups = (NW + G - 1) / G;
        G = (NW + ngroups - 1) / ngroups;
    }
    if (h->batch) G = (G / c.nw_chan > 0 ? G / c.nw_chan : 1) * c.nw_chan;
    h->G = G;
    size_t need = (size_t)G * pb + (G < NW ? pb : 0) + (size_t)ntiles * 4 + (size_t)c.n * 4 +
                  ((p->flags & RICK_UNIFORM_WEIGHT) ? (size_t)c.n * c.n * 4 : 0) + (64u << 20);
    if (need > fr) {
        delete h;
        return RICK_ERR_OOM;
    }
    auto cleanup = [&](rick_status st) {
        snprintf(g_create_error, sizeof(g_create_error), "%s",
                 h->last_error[0] ? h->last_error : rick_status_string(st));
        rick_destroy(h);
        return st;
    };
    if (cudaMalloc(&h->taper, (size_t)c.n * sizeof(float)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
    if (cudaMalloc(&h->planes, (size_t)G * pb) != cudaSuccess) return cleanup(RICK_ERR_OOM);
    if (G < NW && !h->batch && cudaMalloc(&h->acc, pb) != cudaSuccess) return cleanup(RICK_ERR_OOM);
    if (h->batch) {
        std::vector<float2> cw(nchan);
        for (int ch = 0; ch < nchan; ++ch) {
            const double dw = (p->nw > 1) ? (w_max[ch] - w_min[ch]) / p->nw : (w_max[ch] - w_min[ch]);
            cw[ch] = make_float2((float)w_min[ch], (p->nw > 1) ? (float)(1.0 / dw) : 0.0f);
        }
        if (cudaMalloc(&h->chan_w, sizeof(float2) * nchan) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMalloc(&h->chan_off, sizeof(int64_t) * (nchan + 1)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMalloc(&h->chan_sw, sizeof(double) * nchan) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMalloc(&h->chan_scr, sizeof(float4) * nchan) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMalloc(&h->b_off, sizeof(uint32_t) * (ntiles + 1)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (G < NW) {
            // a second plane buffer for pipelined groups, when it fits (else groups run one by one)
            size_t fr2 = 0, tot2 = 0;
            if (cudaMemGetInfo(&fr2, &tot2) == cudaSuccess && (size_t)G * pb + 2 * pb + (256u << 20) < fr2 &&
                cudaMalloc((void**)&h->planes2, (size_t)G * pb) == cudaSuccess) {
                h->bytes_held += (size_t)G * pb;
                if (cudaStreamCreateWithFlags(&h->fft_stream, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess)
                    return cleanup(RICK_ERR_CUDA);
                for (int b = 0; b < 2; ++b)
                    if (cudaEventCreateWithFlags(&h->ev_gridded[b], cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming) != cudaSuccess)
                        return cleanup(RICK_ERR_CUDA);
            }
        }
        if (cudaMemcpy(h->chan_w, cw.data(), sizeof(float2) * nchan, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(RICK_ERR_CUDA);
        // each channel's w-screen constants (w_min + dw/2, dw) as float pairs
        std::vector<float4> cs(nchan);
        for (int ch = 0; ch < nchan; ++ch) {
            const double dw = (p->nw > 1) ? (w_max[ch] - w_min[ch]) / p->nw : (w_max[ch] - w_min[ch]);
            split(w_min[ch] + 0.5 * dw, &cs[ch].x, &cs[ch].y);
            split(dw, &cs[ch].z, &cs[ch].w);
        }
        if (cudaMemcpy(h->chan_scr, cs.data(), sizeof(float4) * nchan, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(RICK_ERR_CUDA);
        h->cfg.chan_w = h->chan_w;
        h->cfg.chan_off = h->chan_off;
    }
    if (cudaMalloc(&h->cursor, (size_t)(ntiles * c.cstride + 1) * sizeof(uint32_t)) != cudaSuccess)
        return cleanup(RICK_ERR_OOM);
    if (cudaMalloc(&h->block_sums, scan_block_sums_len(ntiles) * sizeof(uint32_t)) != cudaSuccess)
        return cleanup(RICK_ERR_OOM);
    if (cudaMalloc(&h->ctr, sizeof(Counters)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
    {
        const double one = 1.0;
        if (cudaMalloc((void**)&h->one, sizeof(double)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMemcpy(h->one, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(RICK_ERR_CUDA);
    }
    if (p->flags & RICK_UNIFORM_WEIGHT) {
        if (cudaMalloc(&h->density, (size_t)c.n * c.n * sizeof(uint32_t)) != cudaSuccess)
            return cleanup(RICK_ERR_OOM);
        if (cudaMemset(h->density, 0, (size_t)c.n * c.n * sizeof(uint32_t)) != cudaSuccess)
            return cleanup(RICK_ERR_CUDA);
    }
    h->bytes_held = (size_t)c.n * 4 + (size_t)G * pb + (h->acc ? pb : 0) + (size_t)ntiles * 4 * (h->batch ? 2 : 1) +
                    scan_block_sums_len(ntiles) * 4 + sizeof(Counters) +
                    ((p->flags & RICK_UNIFORM_WEIGHT) ? (size_t)c.n * c.n * 4 : 0);
    if (cudaMemset(h->ctr, 0, sizeof(Counters)) != cudaSuccess) return cleanup(RICK_ERR_CUDA);
    if (launch_taper(c, h->kernel_param, h->taper, nullptr) != cudaSuccess) return cleanup(RICK_ERR_CUDA);
    if (c.Sw > 1) {
        // -(n - 1) over the image reaches its largest value at the corners
        const double half = 0.5 * p->n * p->pixel_rad, r2 = 2.0 * half * half;
        const double umax = r2 >= 1.0 ? 1.0 : r2 / (1.0 + std::sqrt(1.0 - r2));
        const double dw = (p->w_max - p->w_min) / p->nw;
        if (cudaMalloc((void**)&h->wcorr, sizeof(float) * kWcorrLen) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (launch_wcorr(c, dw * umax, kWcorrLen, h->wcorr, nullptr) != cudaSuccess) return cleanup(RICK_ERR_CUDA);
        h->wc_scale = (float)((kWcorrLen - 1) / umax);
        // beyond the w-kernel's passband the correction divides by ~0: refuse
        std::vector<float> tab(kWcorrLen);
        if (cudaMemcpy(tab.data(), h->wcorr, sizeof(float) * kWcorrLen, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cleanup(RICK_ERR_CUDA);
        float lo = tab[0];
        for (float x : tab) lo = x < lo ? x : lo;
        if (!(lo >= kMinWcorr)) {
            snprintf(h->last_error, sizeof(h->last_error),
                     "w_support %d: the grid correction in w falls to %.3g in the image (dw (1 - n) = %.3g "
                     "plane widths at the corners is beyond the kernel's passband): use more w-planes",
                     c.Sw, (double)lo, dw * umax);
            return cleanup(RICK_ERR_ARG);
        }
    }
    {
        // kernel tap polynomials: fitted on the device, carried in the kernel parameters
        float* d_coef = nullptr;
        double* d_err = nullptr;
        float coef[kMaxSupport * kPolyTerms];
        double err[kMaxSupport];
        if (cudaMalloc(&d_coef, sizeof(coef)) != cudaSuccess) return cleanup(RICK_ERR_OOM);
        if (cudaMalloc(&d_err, sizeof(err)) != cudaSuccess) {
            cudaFree(d_coef);
            return cleanup(RICK_ERR_OOM);
        }
        cudaError_t e = launch_fit_taps(c, h->kernel_param, d_coef, d_err, nullptr);
        if (e == cudaSuccess) e = cudaMemcpy(coef, d_coef, sizeof(coef), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(err, d_err, sizeof(err), cudaMemcpyDeviceToHost);
        cudaFree(d_coef);
        cudaFree(d_err);
        if (e != cudaSuccess) return cleanup(RICK_ERR_CUDA);
        double worst = 0.0;
        for (int t = 0; t < c.S; ++t) worst = err[t] > worst ? err[t] : worst;
        if (!(worst <= 2e-6)) {  // kernel too sharp for degree-10 taps
            snprintf(h->last_error, sizeof(h->last_error),
                     "kernel taps: the degree-10 polynomial fit misses the kernel by %.3g (> 2e-6): the kernel is "
                     "too sharp for support %d (widen kernel_param)", worst, c.S);
            return cleanup(RICK_ERR_ARG);
        }
        for (int t = 0; t < kMaxSupport; ++t)
            for (int j = 0; j < kPolyTerms; ++j) h->cfg.coef[t][j] = (t < c.S) ? coef[t * kPolyTerms + j] : 0.0f;
        set_tap_sum(h->cfg);
    }
    // the cuFFT plans this handle's transform path uses
    {
        cufftHandle plan;
        int n1 = 0, n2 = 0;
        // batches take the split from n = 1024 on (one row plan, one
        // k_colfft launch per group and a fused stack per channel)
        h->batch_split = h->batch && colstack_shape(p->n, &n1, &n2) && p->n >= kBatchSplitMinN &&
                         !(p->flags & RICK_FFT_2D);
        const bool split = h->batch ? h->batch_split : use_split(*p, &n1, &n2);
        const int kind = split ? kPlanRows : kPlan2D;
        // the split keeps the handle's planes in b-major row order
        h->cfg.row_perm = 0;
        if (split)
            while ((1 << h->cfg.row_perm) < n1) ++h->cfg.row_perm;
        s = get_plan(h, G, &plan, kind);
        if (s) return cleanup(s);
        if (NW % G) {
            s = get_plan(h, NW % G, &plan, kind);
            if (s) return cleanup(s);
        }
    }
    if (h->batch_split) {
        // twiddles and tensor maps of both plane buffers, outside any capture
        s = colfft_ready(h);
        if (s) return cleanup(s);
        if (encode_colstack_map(h->colmap, h->planes, p->n, h->G) != cudaSuccess) return cleanup(RICK_ERR_CUDA);
        h->colmap_ready = true;
        if (h->planes2 && (encode_colstack_map(h->colmap2, h->planes2, p->n, h->G) != cudaSuccess ||
                           encode_colfft_map(h->cfmap2, h->planes2, p->n, h->G) != cudaSuccess))
            return cleanup(RICK_ERR_CUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return cleanup(RICK_ERR_CUDA);
    *out = h;
    return RICK_OK;
}

rick_status rick_create(const rick_params* p, rick_handle* out)
{
    return create_impl(p, 1, nullptr, nullptr, out);
}

static void async_release(rick_handle h);

rick_status rick_destroy(rick_handle h)
{
    if (!h) return RICK_OK;
    cudaStreamSynchronize(h->stream);
    async_release(h);
    free_chunks(h);
    cudaStreamSynchronize(h->stream);
    for (auto& kv : h->plans) cufftDestroy(kv.second);
    resolve_timer(h, false);
    for (auto& ev : h->timer.spare) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    cudaFree(h->taper);
    cudaFree(h->cf_tw);
    cudaFree(h->sw_dev);
    cudaFree(h->planes);
    cudaFree(h->acc);
    cudaFree(h->cursor);
    cudaFree(h->block_sums);
    cudaFree(h->density);
    cudaFree(h->ctr);
    cudaFree(h->one);
    cudaFree(h->wcorr);
    cudaFree(h->fft_work);
    cudaFree(h->stage);
    cudaFree(h->img_dev);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    cudaFree(h->chan_w);
    cudaFree(h->chan_off);
    cudaFree(h->chan_sw);
    cudaFree(h->chan_scr);
    cudaFree(h->b_off);
    cudaFree(h->b_ent);
    cudaFree(h->b_heavy);
    if (h->planes2) {
        if (h->fft_stream) cudaStreamSynchronize(h->fft_stream);
        cudaFree(h->planes2);
    }
    if (h->fft_stream) cudaStreamDestroy(h->fft_stream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_gridded[b]) cudaEventDestroy(h->ev_gridded[b]);
        if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
    }
    if (h->pool) cudaMemPoolDestroy(h->pool);
    delete h;
    return RICK_OK;
}

rick_status rick_set_stream(rick_handle h, void* cuda_stream)
{
    if (!h) return RICK_ERR_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    for (auto& kv : h->plans) RICK_FFT(h, cufftSetStream(kv.second, h->stream));
    return RICK_OK;
}

rick_status rick_reset(rick_handle h)
{
    if (!h) return RICK_ERR_ARG;
    free_chunks(h);
    RICK_CU(h, cudaMemsetAsync(h->ctr, 0, sizeof(Counters), h->stream));
    if (h->density)
        RICK_CU(h, cudaMemsetAsync(h->density, 0, (size_t)h->cfg.n * h->cfg.n * sizeof(uint32_t), h->stream));
    h->density_frozen = false;
    h->user_density = false;
    return RICK_OK;
}

rick_status rick_add_density(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                             const float* weights, int64_t nvis)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    rick_status s = check_vis_args(h, vis, u, v, w, nvis);
    if (s) return s;
    if (!h->density) return fail(h, RICK_ERR_STATE, "uniform weighting is not enabled for this handle");
    if (h->density_frozen) return fail(h, RICK_ERR_STATE, "density is frozen once rick_grid has run; reset first");
    RICK_CU(h, launch_density(h->cfg, u, v, w, weights, reinterpret_cast<const float2*>(vis), nvis, h->density,
                              h->stream));
    h->user_density = true;
    return RICK_OK;
}

rick_status rick_grid(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                      const float* weights, int64_t nvis)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    rick_status s = check_vis_args(h, vis, u, v, w, nvis);
    if (s) return s;
    if (nvis == 0) return RICK_OK;
    const GridCfg& c = h->cfg;
    const float2* vis2 = reinterpret_cast<const float2*>(vis);
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    const int64_t cap = entries_bound(c, nvis);
    const size_t off_bytes = (size_t)(ntiles + 1) * sizeof(uint32_t);
    const size_t ent_bytes = (size_t)cap * sizeof(float4);
    if ((uint64_t)cap > 0xffffffffULL) return fail(h, RICK_ERR_ARG, "too many entries for one chunk");
    size_t fr = 0, tot = 0;
    RICK_CU(h, cudaMemGetInfo(&fr, &tot));
    if (off_bytes + ent_bytes + (64u << 20) > fr)
        return fail(h, RICK_ERR_OOM, "chunk of %lld measurements needs %zu bytes, %zu free", (long long)nvis,
                    off_bytes + ent_bytes, fr);
    PhaseScope scope(h, kPhasePrep);
    if (h->density && !h->density_frozen && !h->user_density) {
        RICK_CU(h, launch_density(c, u, v, w, weights, vis2, nvis, h->density, h->stream));
        count_launches(h, 1);
    }
    h->density_frozen = true;
    rick_imager::Chunk ch{};
    ch.cap = cap;
    RICK_CU(h, cudaMallocFromPoolAsync((void**)&ch.off, off_bytes, h->pool, h->stream));
    cudaError_t e = cudaMallocFromPoolAsync((void**)&ch.ent, ent_bytes, h->pool, h->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(ch.off, h->stream);
        return fail(h, RICK_ERR_OOM, "cudaMallocFromPoolAsync(entries): %s", cudaGetErrorString(e));
    }
    // the chunk is registered only once every kernel that fills it is enqueued,
    // so a failed call never leaves unfilled offsets for the gridder to read
    e = cudaMemsetAsync(h->cursor, 0, (size_t)ntiles * c.cstride * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = launch_count(c, u, v, w, weights, vis2, nvis, h->cursor, h->stream);
    if (e == cudaSuccess)
        e = launch_scan(h->cursor, ntiles, c.cstride, ch.off, h->cursor, h->block_sums, h->stream);
    if (e == cudaSuccess)
        e = launch_scatter(c, u, v, w, weights, vis2, nvis, h->density, h->cursor, ch.ent, h->ctr, nullptr,
                           h->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(ch.off, h->stream);
        cudaFreeAsync(ch.ent, h->stream);
        return fail(h, RICK_ERR_CUDA, "rick_grid launch: %s", cudaGetErrorString(e));
    }
    h->chunks.push_back(ch);
    h->bytes_held += off_bytes + ent_bytes;
    count_launches(h, 5);
    return RICK_OK;
}

rick_status rick_grid_planes(rick_handle h, int32_t k0, int32_t nk, float* planes)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    if (k0 < 0 || nk < 0 || k0 + nk > h->p.nw) return fail(h, RICK_ERR_ARG, "plane range out of bounds");
    if (nk == 0) return RICK_OK;
    if (!planes) return fail(h, RICK_ERR_ARG, "planes is NULL");
    return grid_pass(h, k0, nk, false, reinterpret_cast<float2*>(planes), true);
}

rick_status rick_fft_and_stack(rick_handle h, float* image)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    if (!image) return fail(h, RICK_ERR_ARG, "image is NULL");
    const rick_params& p = h->p;
    const double dw = (p.nw > 1) ? (p.w_max - p.w_min) / p.nw : (p.w_max - p.w_min);
    StackArgs a{};
    a.n = p.n;
    split(p.pixel_rad * p.pixel_rad, &a.dl2_hi, &a.dl2_lo);
    split(p.w_min + 0.5 * dw, &a.wb_hi, &a.wb_lo);
    split(dw, &a.dw_hi, &a.dw_lo);
    a.flags = p.flags;
    a.wcorr = h->cfg.Sw > 1 ? h->wcorr : nullptr;
    a.wc_scale = h->wc_scale;
    a.wait_ns = h->dbg_wait_ns;
    a.skip_slot1 = h->dbg_skip_slot1;
    // the split (use_split): cuFFT transforms the rows, k_colfft the first
    // factor of the columns, k_colstack the last factor with the screen and
    // the stack (planes in b-major row order, GridCfg::row_perm); otherwise
    // cuFFT's 2D plan and k_stack
    int n1 = 0, n2 = 0;
    const bool split = use_split(p, &n1, &n2);
    const int lo = h->cfg.plane_lo, hi = h->cfg.plane_hi;
    for (int k0 = lo; k0 < hi; k0 += h->G) {
        const int nk = (hi - k0 < h->G) ? hi - k0 : h->G;
        rick_status s = grid_pass(h, k0, nk, true, h->planes);
        if (s) return s;
        cufftComplex* planes = reinterpret_cast<cufftComplex*>(h->planes);
        a.k0 = k0;
        a.nk = nk;
        a.first = (k0 == lo);
        a.last = (k0 + nk >= hi);
        if (split) {
            cufftHandle rows;
            if ((s = get_plan(h, nk, &rows, kPlanRows))) return s;
            if ((s = colfft_ready(h))) return s;
            {
                PhaseScope fs(h, kPhaseFft);
                RICK_FFT(h, cufftExecC2C(rows, planes, planes, CUFFT_INVERSE));
            }
            {
                PhaseScope cs(h, kPhaseColfft);
                RICK_CU(h, launch_colfft(h->cfmap, h->cf_tw, h->planes, p.n, nk, +1, h->dbg_wait_ns, &h->ctr->err,
                                         h->stream));
                count_launches(h, 1);
            }
            if (!h->colmap_ready) {
                RICK_CU(h, encode_colstack_map(h->colmap, h->planes, p.n, h->G));
                h->colmap_ready = true;
            }
            PhaseScope ss(h, kPhaseStack);
            RICK_CU(h, launch_colstack(h->colmap, a, n1, n2, h->acc, h->taper, norm_sum(h), image, &h->ctr->err,
                                       h->stream));
        } else {
            cufftHandle plan;
            if ((s = get_plan(h, nk, &plan))) return s;
            {
                PhaseScope fs(h, kPhaseFft);
                RICK_FFT(h, cufftExecC2C(plan, planes, planes, CUFFT_INVERSE));
            }
            PhaseScope ss(h, kPhaseStack);
            RICK_CU(h, launch_stack(a, h->planes, h->acc, h->taper, norm_sum(h), image, h->stream));
        }
        count_launches(h, 1);
    }
    return RICK_OK;
}

// The degridding chain shared by rick_degrid and rick_predict: sort the
// measurements by the tile of their first footprint cell, then per plane
// group spread the image (adjoint of the finalisation with the weight sum at
// *sum_w, conjugate w-screen), transform forward and gather each footprint
// with the gridding taps, times the weight (density: uniform weighting).
static rick_status degrid_impl(rick_handle h, const GridCfg& c, const double* sum_w, const uint32_t* density,
                               const float* image_grad, const float* u, const float* v, const float* w,
                               const float* weights, int64_t nvis, float* vis_grad)
{
    const rick_params& p = h->p;
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    const size_t off_bytes = (size_t)(ntiles + 1) * sizeof(uint32_t);
    const size_t perm_bytes = (size_t)nvis * sizeof(uint32_t);
    size_t fr = 0, tot = 0;
    RICK_CU(h, cudaMemGetInfo(&fr, &tot));
    if (off_bytes + perm_bytes + (64u << 20) > fr) return fail(h, RICK_ERR_OOM, "degrid scratch does not fit");
    PhaseScope scope(h, kPhaseDegrid);
    uint32_t* off = nullptr;
    uint32_t* perm = nullptr;
    RICK_CU(h, cudaMallocFromPoolAsync((void**)&off, off_bytes, h->pool, h->stream));
    cudaError_t e = cudaMallocFromPoolAsync((void**)&perm, perm_bytes, h->pool, h->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(off, h->stream);
        return fail(h, RICK_ERR_OOM, "cudaMallocFromPoolAsync(perm): %s", cudaGetErrorString(e));
    }
    float2* grad = reinterpret_cast<float2*>(vis_grad);
    const double dw = (p.nw > 1) ? (p.w_max - p.w_min) / p.nw : (p.w_max - p.w_min);
    StackArgs a{};
    a.n = p.n;
    split(p.pixel_rad * p.pixel_rad, &a.dl2_hi, &a.dl2_lo);
    split(p.w_min + 0.5 * dw, &a.wb_hi, &a.wb_lo);
    split(dw, &a.dw_hi, &a.dw_lo);
    a.flags = p.flags;
    a.wcorr = h->cfg.Sw > 1 ? h->wcorr : nullptr;
    a.wc_scale = h->wc_scale;
    rick_status st = RICK_OK;
    e = cudaMemsetAsync(grad, 0, (size_t)nvis * sizeof(float2), h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->cursor, 0, (size_t)ntiles * c.cstride * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = launch_primary_count(c, u, v, w, weights, nvis, h->cursor, h->stream);
    if (e == cudaSuccess) e = launch_scan(h->cursor, ntiles, c.cstride, off, h->cursor, h->block_sums, h->stream);
    if (e == cudaSuccess) e = launch_primary_scatter(c, u, v, w, weights, nvis, h->cursor, perm, h->stream);
    if (e != cudaSuccess) st = fail(h, RICK_ERR_CUDA, "rick_degrid sort: %s", cudaGetErrorString(e));
    if (!st) count_launches(h, 5);
    // the adjoint of rick_fft_and_stack's transform path: with the split,
    // k_spreadcol writes the planes after the adjoint of the last column
    // factor, then k_colfft's forward first column factor and cuFFT's forward
    // rows; otherwise k_spread and cuFFT's forward 2D plan
    int n1 = 0, n2 = 0;
    const bool split = use_split(p, &n1, &n2);
    cufftComplex* planes = reinterpret_cast<cufftComplex*>(h->planes);
    for (int k0 = c.plane_lo; !st && k0 < c.plane_hi; k0 += h->G) {
        const int nk = (c.plane_hi - k0 < h->G) ? c.plane_hi - k0 : h->G;
        a.k0 = k0;
        a.nk = nk;
        e = split ? launch_spreadcol(a, n1, n2, image_grad, h->taper, sum_w, h->planes, h->stream)
                  : launch_spread(a, image_grad, h->taper, sum_w, h->planes, h->stream);
        if (e != cudaSuccess) {
            st = fail(h, RICK_ERR_CUDA, "%s: %s", split ? "k_spreadcol" : "k_spread", cudaGetErrorString(e));
            break;
        }
        cufftResult r = CUFFT_SUCCESS;
        if (split) {
            cufftHandle rows;
            if ((st = get_plan(h, nk, &rows, kPlanRows))) break;
            if ((st = colfft_ready(h))) break;
            e = launch_colfft(h->cfmap, h->cf_tw, h->planes, p.n, nk, -1, h->dbg_wait_ns, &h->ctr->err, h->stream);
            if (e != cudaSuccess) {
                st = fail(h, RICK_ERR_CUDA, "k_colfft: %s", cudaGetErrorString(e));
                break;
            }
            count_launches(h, 1);
            r = cufftExecC2C(rows, planes, planes, CUFFT_FORWARD);
        } else {
            cufftHandle plan;
            if ((st = get_plan(h, nk, &plan))) break;
            r = cufftExecC2C(plan, planes, planes, CUFFT_FORWARD);
        }
        if (r != CUFFT_SUCCESS) {
            st = fail(h, RICK_ERR_CUFFT, "cufftExecC2C(FORWARD): error %d", (int)r);
            break;
        }
        e = launch_degrid_gather(c, perm, off, k0, nk, h->planes, u, v, w, weights, density, grad, h->stream);
        if (e != cudaSuccess) {
            st = fail(h, RICK_ERR_CUDA, "k_degrid_gather: %s", cudaGetErrorString(e));
            break;
        }
        count_launches(h, 2);
    }
    cudaFreeAsync(off, h->stream);
    cudaFreeAsync(perm, h->stream);
    return st;
}

rick_status rick_degrid(rick_handle h, const float* image_grad, const float* u, const float* v, const float* w,
                        const float* weights, int64_t nvis, float* vis_grad)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: the adjoint is single-channel");
    if (nvis < 0) return fail(h, RICK_ERR_ARG, "nvis must be >= 0");
    if (nvis > ((int64_t)1 << 30)) return fail(h, RICK_ERR_ARG, "at most 2^30 measurements per call");
    if (nvis > 0 && (!u || !v || !w || !vis_grad)) return fail(h, RICK_ERR_ARG, "u, v, w, vis_grad must not be NULL");
    if (!image_grad) return fail(h, RICK_ERR_ARG, "image_grad is NULL");
    if (h->chunks.empty())
        return fail(h, RICK_ERR_STATE, "rick_degrid needs the weight sum of a forward pass: call rick_grid first");
    if (nvis == 0) return RICK_OK;
    return degrid_impl(h, h->cfg, norm_sum(h), h->density, image_grad, u, v, w, weights, nvis, vis_grad);
}

rick_status rick_predict(rick_handle h, const float* model, const float* u, const float* v, const float* w,
                         int64_t nvis, float* vis)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: prediction is single-channel");
    if (nvis < 0) return fail(h, RICK_ERR_ARG, "nvis must be >= 0");
    if (nvis > ((int64_t)1 << 30)) return fail(h, RICK_ERR_ARG, "at most 2^30 measurements per call");
    if (nvis > 0 && (!u || !v || !w || !vis)) return fail(h, RICK_ERR_ARG, "u, v, w, vis must not be NULL");
    if (!model) return fail(h, RICK_ERR_ARG, "model is NULL");
    if (nvis == 0) return RICK_OK;
    GridCfg c = h->cfg;
    c.uniform = 0;  // unit weights, no density
    return degrid_impl(h, c, h->one, nullptr, model, u, v, w, nullptr, nvis, vis);
}


rick_status rick_image_host(rick_handle h, const float* vis_host, const float* u_host, const float* v_host,
                            const float* w_host, const float* weights_host, int64_t nvis, float* image_host)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    rick_status s = check_vis_args(h, vis_host, u_host, v_host, w_host, nvis);
    if (s) return s;
    if (!image_host) return fail(h, RICK_ERR_ARG, "image_host is NULL");
    const size_t per = (weights_host ? 6 : 5) * sizeof(float);
    const size_t need = (size_t)nvis * per;
    if (need > h->stage_bytes) {
        RICK_CU(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->stage);
        h->bytes_held -= h->stage_bytes;
        h->stage = nullptr;
        h->stage_bytes = 0;
        RICK_CU(h, cudaMalloc((void**)&h->stage, need));
        h->stage_bytes = need;
        h->bytes_held += need;
    }
    const size_t img = (size_t)h->p.n * h->p.n * ((h->p.flags & RICK_REAL_IMAGE) ? 1 : 2) * sizeof(float);
    if (img > h->img_bytes) {
        RICK_CU(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->img_dev);
        h->bytes_held -= h->img_bytes;
        h->img_dev = nullptr;
        h->img_bytes = 0;
        RICK_CU(h, cudaMalloc((void**)&h->img_dev, img));
        h->img_bytes = img;
        h->bytes_held += img;
    }
    float* d_vis = h->stage;
    float* d_u = d_vis + 2 * nvis;
    float* d_v = d_u + nvis;
    float* d_w = d_v + nvis;
    float* d_wt = weights_host ? d_w + nvis : nullptr;
    const size_t fb = (size_t)nvis * sizeof(float);
    RICK_CU(h, cudaMemcpyAsync(d_vis, vis_host, 2 * fb, cudaMemcpyHostToDevice, h->stream));
    RICK_CU(h, cudaMemcpyAsync(d_u, u_host, fb, cudaMemcpyHostToDevice, h->stream));
    RICK_CU(h, cudaMemcpyAsync(d_v, v_host, fb, cudaMemcpyHostToDevice, h->stream));
    RICK_CU(h, cudaMemcpyAsync(d_w, w_host, fb, cudaMemcpyHostToDevice, h->stream));
    if (d_wt) RICK_CU(h, cudaMemcpyAsync(d_wt, weights_host, fb, cudaMemcpyHostToDevice, h->stream));
    s = rick_reset(h);
    if (s) return s;
    s = rick_grid(h, d_vis, d_u, d_v, d_w, d_wt, nvis);
    if (s) return s;
    s = rick_fft_and_stack(h, h->img_dev);
    if (s) return s;
    RICK_CU(h, cudaMemcpyAsync(image_host, h->img_dev, img, cudaMemcpyDeviceToHost, h->stream));
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    return RICK_OK;
}

static rick_status async_init(rick_handle h)
{
    if (h->async_ready) return RICK_OK;
    RICK_CU(h, cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
    RICK_CU(h, cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        RICK_CU(h, cudaEventCreateWithFlags(&h->ev_staged[b], cudaEventDisableTiming));
        RICK_CU(h, cudaEventCreateWithFlags(&h->ev_computed[b], cudaEventDisableTiming));
        RICK_CU(h, cudaEventCreateWithFlags(&h->ev_fetched[b], cudaEventDisableTiming));
    }
    h->async_ready = true;
    return RICK_OK;
}

static void async_release(rick_handle h)
{
    if (!h->async_ready) return;
    cudaStreamSynchronize(h->h2d);
    cudaStreamSynchronize(h->d2h);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->astage[b]);
        cudaFree(h->aimg[b]);
        cudaEventDestroy(h->ev_staged[b]);
        cudaEventDestroy(h->ev_computed[b]);
        cudaEventDestroy(h->ev_fetched[b]);
    }
    cudaStreamDestroy(h->h2d);
    cudaStreamDestroy(h->d2h);
    h->async_ready = false;
}

rick_status rick_image_host_async(rick_handle h, const float* vis_host, const float* u_host, const float* v_host,
                                  const float* w_host, const float* weights_host, int64_t nvis, float* image_host)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: use rick_image_batch");
    rick_status s = check_vis_args(h, vis_host, u_host, v_host, w_host, nvis);
    if (s) return s;
    if (!image_host) return fail(h, RICK_ERR_ARG, "image_host is NULL");
    if ((s = async_init(h))) return s;
    const size_t fb = (size_t)nvis * sizeof(float);
    const size_t need = (weights_host ? 6 : 5) * fb;
    const size_t img = (size_t)h->p.n * h->p.n * ((h->p.flags & RICK_REAL_IMAGE) ? 1 : 2) * sizeof(float);
    if (need > h->astage_bytes || img > h->aimg_bytes) {
        // grow both slots once nothing is in flight
        RICK_CU(h, cudaStreamSynchronize(h->h2d));
        RICK_CU(h, cudaStreamSynchronize(h->stream));
        RICK_CU(h, cudaStreamSynchronize(h->d2h));
        const size_t sb = need > h->astage_bytes ? need : h->astage_bytes;
        const size_t ib = img > h->aimg_bytes ? img : h->aimg_bytes;
        for (int b = 0; b < 2; ++b) {
            cudaFree(h->astage[b]);
            cudaFree(h->aimg[b]);
            h->astage[b] = nullptr;
            h->aimg[b] = nullptr;
        }
        h->bytes_held -= 2 * (h->astage_bytes + h->aimg_bytes);
        h->astage_bytes = h->aimg_bytes = 0;
        for (int b = 0; b < 2; ++b) {
            RICK_CU(h, cudaMalloc((void**)&h->astage[b], sb));
            RICK_CU(h, cudaMalloc((void**)&h->aimg[b], ib));
        }
        h->astage_bytes = sb;
        h->aimg_bytes = ib;
        h->bytes_held += 2 * (sb + ib);
    }
    const int b = h->aslot;
    h->aslot ^= 1;
    float* d_vis = h->astage[b];
    float* d_u = d_vis + 2 * nvis;
    float* d_v = d_u + nvis;
    float* d_w = d_v + nvis;
    float* d_wt = weights_host ? d_w + nvis : nullptr;
    // upload once the compute that last read this slot is done
    RICK_CU(h, cudaStreamWaitEvent(h->h2d, h->ev_computed[b], 0));
    RICK_CU(h, cudaMemcpyAsync(d_vis, vis_host, 2 * fb, cudaMemcpyHostToDevice, h->h2d));
    RICK_CU(h, cudaMemcpyAsync(d_u, u_host, fb, cudaMemcpyHostToDevice, h->h2d));
    RICK_CU(h, cudaMemcpyAsync(d_v, v_host, fb, cudaMemcpyHostToDevice, h->h2d));
    RICK_CU(h, cudaMemcpyAsync(d_w, w_host, fb, cudaMemcpyHostToDevice, h->h2d));
    if (d_wt) RICK_CU(h, cudaMemcpyAsync(d_wt, weights_host, fb, cudaMemcpyHostToDevice, h->h2d));
    RICK_CU(h, cudaEventRecord(h->ev_staged[b], h->h2d));
    // image once the inputs have landed and the last download of this slot is done
    RICK_CU(h, cudaStreamWaitEvent(h->stream, h->ev_staged[b], 0));
    RICK_CU(h, cudaStreamWaitEvent(h->stream, h->ev_fetched[b], 0));
    if ((s = rick_reset(h))) return s;
    if ((s = rick_grid(h, d_vis, d_u, d_v, d_w, d_wt, nvis))) return s;
    if ((s = rick_fft_and_stack(h, h->aimg[b]))) return s;
    RICK_CU(h, cudaEventRecord(h->ev_computed[b], h->stream));
    RICK_CU(h, cudaStreamWaitEvent(h->d2h, h->ev_computed[b], 0));
    RICK_CU(h, cudaMemcpyAsync(image_host, h->aimg[b], img, cudaMemcpyDeviceToHost, h->d2h));
    RICK_CU(h, cudaEventRecord(h->ev_fetched[b], h->d2h));
    return RICK_OK;
}

rick_status rick_synchronize(rick_handle h)
{
    if (!h) return RICK_ERR_ARG;
    if (h->async_ready) RICK_CU(h, cudaStreamSynchronize(h->h2d));
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    if (h->async_ready) RICK_CU(h, cudaStreamSynchronize(h->d2h));
    return RICK_OK;
}

rick_status rick_set_timing(rick_handle h, int32_t enable)
{
    if (!h) return RICK_ERR_ARG;
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    resolve_timer(h, false);
    for (int ph = 0; ph < kNumPhases; ++ph) {
        h->timer.ms[ph] = 0.0;
        h->timer.calls[ph] = 0;
    }
    h->timer.launches = 0;
    h->timer.on = enable != 0;
    return RICK_OK;
}

rick_status rick_get_timing(rick_handle h, rick_timing* out)
{
    if (!h || !out) return RICK_ERR_ARG;
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    resolve_timer(h, true);
    out->prep_ms = h->timer.ms[kPhasePrep];
    out->grid_ms = h->timer.ms[kPhaseGrid];
    out->fft_ms = h->timer.ms[kPhaseFft];
    out->stack_ms = h->timer.ms[kPhaseStack];
    out->degrid_ms = h->timer.ms[kPhaseDegrid];
    out->prep_calls = h->timer.calls[kPhasePrep];
    out->grid_calls = h->timer.calls[kPhaseGrid];
    out->fft_calls = h->timer.calls[kPhaseFft];
    out->stack_calls = h->timer.calls[kPhaseStack];
    out->degrid_calls = h->timer.calls[kPhaseDegrid];
    out->kernel_launches = h->timer.launches;
    out->colfft_ms = h->timer.ms[kPhaseColfft];
    out->colfft_calls = h->timer.calls[kPhaseColfft];
    return RICK_OK;
}

rick_status rick_create_batch(const rick_params* p, int32_t nchan, const double* w_min, const double* w_max,
                              rick_handle* out)
{
    if (!out || !w_min || !w_max || nchan < 1) return RICK_ERR_ARG;
    return create_impl(p, nchan, w_min, w_max, out);
}

// One batch step: placement + counting sort over all channels, then per plane
// group the gridder, one cuFFT batch and one stack per channel.  Everything it
// enqueues is capturable (no host synchronisation, no allocation).
static rick_status batch_body(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                              const float* weights, int64_t m, float* images)
{
    const GridCfg& c = h->cfg;
    const rick_params& p = h->p;
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    const float2* vis2 = reinterpret_cast<const float2*>(vis);
    {
        PhaseScope scope(h, kPhasePrep);
        RICK_CU(h, cudaMemsetAsync(h->ctr, 0, sizeof(Counters), h->stream));
        RICK_CU(h, cudaMemsetAsync(h->chan_sw, 0, sizeof(double) * h->nchan, h->stream));
        RICK_CU(h, cudaMemsetAsync(h->cursor, 0, (size_t)ntiles * c.cstride * sizeof(uint32_t), h->stream));
        RICK_CU(h, launch_count(c, u, v, w, weights, vis2, m, h->cursor, h->stream));
        RICK_CU(h, launch_scan(h->cursor, ntiles, c.cstride, h->b_off, h->cursor, h->block_sums, h->stream));
        RICK_CU(h, launch_scatter(c, u, v, w, weights, vis2, m, nullptr, h->cursor, h->b_ent, h->ctr, h->chan_sw,
                                  h->stream));
        count_launches(h, 5);
    }
    const size_t img_floats = (size_t)p.n * p.n * ((p.flags & RICK_REAL_IMAGE) ? 1 : 2);
    const size_t nn = (size_t)p.n * p.n;
    // the w-screen constants of channel ch
    auto chan_args = [&](int ch) {
        const double dw = (p.nw > 1) ? (h->chan_wmax[ch] - h->chan_wmin[ch]) / p.nw
                                     : (h->chan_wmax[ch] - h->chan_wmin[ch]);
        StackArgs a{};
        a.n = p.n;
        split(p.pixel_rad * p.pixel_rad, &a.dl2_hi, &a.dl2_lo);
        split(h->chan_wmin[ch] + 0.5 * dw, &a.wb_hi, &a.wb_lo);
        split(dw, &a.dw_hi, &a.dw_lo);
        a.flags = p.flags;
        a.k0 = 0;
        a.nk = c.nw_chan;
        a.first = 1;
        a.last = 1;
        a.wait_ns = h->dbg_wait_ns;
        return a;
    };
    // the split transform of a group in buffer `buf` (b = 0: planes, 1:
    // planes2) on stream st: cuFFT's rows, k_colfft, and per channel the
    // fused last column factor + w-screen + stack (k_colstack)
    auto split_group = [&](float2* buf, int b, int k0, int nk, cudaStream_t st) -> rick_status {
        cufftHandle rows;
        rick_status s = get_plan(h, nk, &rows, kPlanRows);
        if (s) return s;
        int n1 = 0, n2 = 0;
        colstack_shape(p.n, &n1, &n2);
        {
            PhaseScope fs(h, kPhaseFft);
            RICK_FFT(h, cufftSetStream(rows, st));
            RICK_FFT(h, cufftExecC2C(rows, reinterpret_cast<cufftComplex*>(buf), reinterpret_cast<cufftComplex*>(buf),
                                     CUFFT_INVERSE));
        }
        {
            PhaseScope cs(h, kPhaseColfft);
            RICK_CU(h, launch_colfft(b ? h->cfmap2 : h->cfmap, h->cf_tw, buf, p.n, nk, +1, h->dbg_wait_ns,
                                     &h->ctr->err, st));
            count_launches(h, 1);
        }
        // one launch over the group's channels (grid z = channel)
        PhaseScope ss(h, kPhaseStack);
        const int ch0 = k0 / c.nw_chan, nch = nk / c.nw_chan;
        StackArgs a = chan_args(ch0);
        a.plane0 = ch0 * c.nw_chan - k0;
        a.chan_screen = h->chan_scr;
        a.chan0 = ch0;
        a.img_stride = (long long)img_floats;
        RICK_CU(h, launch_colstack(b ? h->colmap2 : h->colmap, a, n1, n2, nullptr, h->taper, h->chan_sw, images,
                                   &h->ctr->err, st, nch));
        count_launches(h, 1);
        return RICK_OK;
    };
    // stack the channels of the group in planes `buf` (first plane k0) on stream st
    auto stack_group = [&](const float2* buf, int k0, int nk, cudaStream_t st) -> rick_status {
        for (int ch = k0 / c.nw_chan; ch < (k0 + nk) / c.nw_chan; ++ch) {
            StackArgs a = chan_args(ch);
            const float2* pl = buf + (size_t)(ch * c.nw_chan - k0) * nn;
            RICK_CU(h, launch_stack(a, pl, nullptr, h->taper, h->chan_sw + ch, images + (size_t)ch * img_floats, st));
            count_launches(h, 1);
        }
        return RICK_OK;
    };
    auto grid_group = [&](float2* buf, int k0, int nk) -> rick_status {
        ChunkList cl{};
        cl.off[0] = h->b_off;
        cl.ent[0] = h->b_ent;
        cl.count = 1;
        RICK_CU(h, launch_grid(c, cl, k0, nk, true, false, h->b_heavy, h->b_heavy_words, buf, h->stream));
        count_launches(h, 2);
        return RICK_OK;
    };
    const bool pipelined = h->planes2 && !h->timer.on && h->G < c.nw;
    if (pipelined) {
        // group g: gridded on the handle's stream into buffer g % 2 (after the
        // stacks of group g - 2 released it), then transformed and stacked on
        // fft_stream, so gridding g + 1 overlaps the FFT and stacks of g
        RICK_CU(h, cudaEventRecord(h->ev_fork, h->stream));
        RICK_CU(h, cudaStreamWaitEvent(h->fft_stream, h->ev_fork, 0));
        int g = 0;
        for (int k0 = 0; k0 < c.nw; k0 += h->G, ++g) {
            const int nk = (c.nw - k0 < h->G) ? c.nw - k0 : h->G;
            const int b = g & 1;
            float2* buf = b ? h->planes2 : h->planes;
            if (g >= 2) RICK_CU(h, cudaStreamWaitEvent(h->stream, h->ev_free[b], 0));
            rick_status s = grid_group(buf, k0, nk);
            if (s) return s;
            RICK_CU(h, cudaEventRecord(h->ev_gridded[b], h->stream));
            RICK_CU(h, cudaStreamWaitEvent(h->fft_stream, h->ev_gridded[b], 0));
            if (h->batch_split) {
                if ((s = split_group(buf, b, k0, nk, h->fft_stream))) return s;
            } else {
                cufftHandle plan;
                if ((s = get_plan(h, nk, &plan))) return s;
                RICK_FFT(h, cufftSetStream(plan, h->fft_stream));
                RICK_FFT(h, cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(buf),
                                         reinterpret_cast<cufftComplex*>(buf), CUFFT_INVERSE));
                if ((s = stack_group(buf, k0, nk, h->fft_stream))) return s;
            }
            RICK_CU(h, cudaEventRecord(h->ev_free[b], h->fft_stream));
        }
        // join: the images are complete on the handle's stream
        RICK_CU(h, cudaStreamWaitEvent(h->stream, h->ev_free[0], 0));
        if (g > 1) RICK_CU(h, cudaStreamWaitEvent(h->stream, h->ev_free[1], 0));
        return RICK_OK;
    }
    for (int k0 = 0; k0 < c.nw; k0 += h->G) {
        const int nk = (c.nw - k0 < h->G) ? c.nw - k0 : h->G;
        {
            PhaseScope scope(h, kPhaseGrid);
            rick_status s = grid_group(h->planes, k0, nk);
            if (s) return s;
        }
        if (h->batch_split) {
            rick_status s = split_group(h->planes, 0, k0, nk, h->stream);
            if (s) return s;
            continue;
        }
        cufftHandle plan;
        rick_status s = get_plan(h, nk, &plan);
        if (s) return s;
        {
            PhaseScope fs(h, kPhaseFft);
            RICK_FFT(h, cufftSetStream(plan, h->stream));
            RICK_FFT(h, cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(h->planes),
                                     reinterpret_cast<cufftComplex*>(h->planes), CUFFT_INVERSE));
        }
        PhaseScope ss(h, kPhaseStack);
        if ((s = stack_group(h->planes, k0, nk, h->stream))) return s;
    }
    return RICK_OK;
}

rick_status rick_image_batch(rick_handle h, const float* vis, const float* u, const float* v, const float* w,
                             const float* weights, const int64_t* chan_offsets, float* images, int32_t use_graph)
{
    if (!h) return RICK_ERR_ARG;
    if (!h->batch) return fail(h, RICK_ERR_STATE, "not a batched handle (rick_create_batch)");
    if (!chan_offsets || !images) return fail(h, RICK_ERR_ARG, "chan_offsets and images must not be NULL");
    if (chan_offsets[0] != 0) return fail(h, RICK_ERR_ARG, "chan_offsets[0] must be 0");
    for (int ch = 0; ch < h->nchan; ++ch)
        if (chan_offsets[ch + 1] < chan_offsets[ch]) return fail(h, RICK_ERR_ARG, "chan_offsets must not decrease");
    const int64_t m = chan_offsets[h->nchan];
    if (m > ((int64_t)1 << 30)) return fail(h, RICK_ERR_ARG, "at most 2^30 measurements per batch");
    if (m > 0 && (!vis || !u || !v || !w)) return fail(h, RICK_ERR_ARG, "vis, u, v, w must not be NULL");
    const GridCfg& c = h->cfg;
    bool stale = false;
    // channel offsets on the device (outside any capture)
    if (h->chan_off_host.size() != (size_t)h->nchan + 1 ||
        memcmp(h->chan_off_host.data(), chan_offsets, sizeof(int64_t) * (h->nchan + 1)) != 0) {
        h->chan_off_host.assign(chan_offsets, chan_offsets + h->nchan + 1);
        RICK_CU(h, cudaMemcpyAsync(h->chan_off, h->chan_off_host.data(), sizeof(int64_t) * (h->nchan + 1),
                                   cudaMemcpyHostToDevice, h->stream));
        RICK_CU(h, cudaStreamSynchronize(h->stream));
        stale = true;
    }
    const int64_t cap = entries_bound(c, m);
    if (cap > h->b_cap) {
        size_t fr = 0, tot = 0;
        RICK_CU(h, cudaMemGetInfo(&fr, &tot));
        if ((size_t)cap * sizeof(float4) + (64u << 20) > fr)
            return fail(h, RICK_ERR_OOM, "batch of %lld measurements needs %zu bytes of entries", (long long)m,
                        (size_t)cap * sizeof(float4));
        RICK_CU(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->b_ent);
        h->b_ent = nullptr;
        h->bytes_held -= (size_t)h->b_cap * sizeof(float4);
        h->b_cap = 0;
        cudaFree(h->b_heavy);
        h->b_heavy = nullptr;
        h->bytes_held -= h->b_heavy_words * sizeof(uint32_t);
        h->b_heavy_words = 0;
        RICK_CU(h, cudaMalloc((void**)&h->b_ent, (size_t)cap * sizeof(float4)));
        h->b_cap = cap;
        const size_t hw = heavy_words_for(cap);
        RICK_CU(h, cudaMalloc((void**)&h->b_heavy, hw * sizeof(uint32_t)));
        h->b_heavy_words = hw;
        h->bytes_held += hw * sizeof(uint32_t);
        h->bytes_held += (size_t)cap * sizeof(float4);
        stale = true;
    }
    if (m == 0) {
        const size_t img = (size_t)h->nchan * h->p.n * h->p.n * ((h->p.flags & RICK_REAL_IMAGE) ? 1 : 2);
        RICK_CU(h, cudaMemsetAsync(images, 0, img * sizeof(float), h->stream));
        return RICK_OK;
    }
    const void* key[7] = {vis, u, v, w, weights, images, (const void*)(intptr_t)m};
    if (use_graph && h->stream == nullptr)
        return fail(h, RICK_ERR_ARG, "graph mode needs a non-default stream (rick_set_stream)");
    if (use_graph && h->graph && !stale && h->graph_m == m && memcmp(key, h->graph_key, sizeof(key)) == 0) {
        RICK_CU(h, cudaGraphLaunch(h->graph, h->stream));
        // per plane group the two gridder kernels, then k_colfft and one
        // k_colstack over its channels (split) or one k_stack per channel
        const int groups = (c.nw + h->G - 1) / h->G;
        count_launches(h, 5 + (h->batch_split ? 4 * groups : 2 * groups + h->nchan));
        return RICK_OK;
    }
    if (!use_graph) return batch_body(h, vis, u, v, w, weights, m, images);
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    const bool timing = h->timer.on;
    h->timer.on = false;  // events are not recorded inside the captured graph
    RICK_CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rick_status s = batch_body(h, vis, u, v, w, weights, m, images);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->timer.on = timing;
    if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return fail(h, RICK_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, RICK_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    memcpy(h->graph_key, key, sizeof(key));
    h->graph_m = m;
    RICK_CU(h, cudaGraphLaunch(h->graph, h->stream));
    return RICK_OK;
}

rick_status rick_set_prep_blocks(rick_handle h, int32_t blocks_per_sm)
{
    if (!h) return RICK_ERR_ARG;
    if (blocks_per_sm < 0 || blocks_per_sm > 64)
        return fail(h, RICK_ERR_ARG, "blocks_per_sm must be in [0, 64] (got %d)", (int)blocks_per_sm);
    h->cfg.prep_bpsm = blocks_per_sm;
    if (h->graph) {  // the captured step holds the old launch shape
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return RICK_OK;
}

// The median of `reps` timed batch steps of handle h on stream st (after one
// untimed step), or a negative value when a step fails.
static double time_batch(rick_handle h, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, const float* vis,
                         const float* u, const float* v, const float* w, const float* weights,
                         const int64_t* chan_offsets, float* images, int reps)
{
    if (rick_image_batch(h, vis, u, v, w, weights, chan_offsets, images, 0) != RICK_OK) return -1.0;
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess ||
            rick_image_batch(h, vis, u, v, w, weights, chan_offsets, images, 0) != RICK_OK ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return -1.0;
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

rick_status rick_autotune_batch(const rick_params* p, int32_t nchan, const double* w_min, const double* w_max,
                                const float* vis, const float* u, const float* v, const float* w,
                                const float* weights, const int64_t* chan_offsets, int32_t* tile_out,
                                int32_t* plane_group_out, int32_t* prep_blocks_out, double* ms_out)
{
    if (!p || !tile_out || !plane_group_out || !chan_offsets || nchan < 1) return RICK_ERR_ARG;
    const int64_t m = chan_offsets[nchan];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return RICK_ERR_CUDA;
    char devname[64];
    snprintf(devname, sizeof(devname), "%s", prop.name);
    for (char* q = devname; *q; ++q)
        if (*q == ' ' || *q == '|') *q = '_';
    // the key names the device and this build of the library, so a cache
    // file never carries a choice across GPUs or library versions
    char key[384];
    snprintf(key, sizeof(key),
             "batch dev=%s sms=%d build=%s_%s n=%d nw=%d nchan=%d S=%d kernel=%d flags=%u m_log2=%d", devname,
             prop.multiProcessorCount, __DATE__, __TIME__, p->n, p->nw, nchan, p->support, p->kernel, p->flags,
             m > 0 ? (int)std::log2((double)m) : 0);
    for (char* q = key; *q; ++q)
        if (*q == '|') *q = '_';
    const char* cache = getenv("RICK_AUTOTUNE_CACHE");
    if (cache && *cache) {
        FILE* f = fopen(cache, "r");
        if (f) {
            char line[640];
            while (fgets(line, sizeof(line), f)) {
                int t = 0, g = 0, pb = 0;
                double ms = 0.0;
                const size_t kl = strlen(key);
                if (strncmp(line, key, kl) == 0 && line[kl] == '|' &&
                    sscanf(line + kl + 1, "%d %d %d %lf", &t, &g, &pb, &ms) == 4) {
                    *tile_out = t;
                    *plane_group_out = g;
                    if (prep_blocks_out) *prep_blocks_out = pb;
                    if (ms_out) *ms_out = ms;
                    fclose(f);
                    return RICK_OK;
                }
            }
            fclose(f);
        }
    }
    const size_t img = (size_t)nchan * p->n * p->n * ((p->flags & RICK_REAL_IMAGE) ? 1 : 2) * sizeof(float);
    float* images = nullptr;
    if (cudaMalloc(&images, img) != cudaSuccess) return RICK_ERR_OOM;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(images);
        return RICK_ERR_CUDA;
    }
    constexpr int kReps = 3;
    double best = 1e30;
    int best_t = 0, best_g = 0, best_pb = 0;
    const int tiles[3] = {16, 32, 64};
    // stage 1: tile side x plane group, each the median of kReps steps
    for (int ti = 0; ti < 3; ++ti) {
        if (tiles[ti] < p->support) continue;
        // plane groups of all channels, half and a quarter of them (with two or
        // more groups the groups are pipelined: gridding overlaps the FFT)
        for (int part = 0; part < 3; ++part) {
            const int div = 1 << part;
            if (part && nchan < div) continue;
            rick_params q = *p;
            q.tile = tiles[ti];
            q.plane_group = part ? (nchan / div) * p->nw : 0;
            rick_handle h = nullptr;
            if (create_impl(&q, nchan, w_min, w_max, &h) != RICK_OK) continue;
            rick_set_stream(h, st);
            const double ms = time_batch(h, st, e0, e1, vis, u, v, w, weights, chan_offsets, images, kReps);
            const int g = h->G;
            rick_destroy(h);
            if (ms > 0.0 && ms < best) {
                best = ms;
                best_t = tiles[ti];
                best_g = g;
            }
        }
    }
    // stage 2: measurements per block of the sort kernels (blocks per SM),
    // on the best tile and plane group
    if (best_t) {
        rick_params q = *p;
        q.tile = best_t;
        q.plane_group = best_g;
        rick_handle h = nullptr;
        if (create_impl(&q, nchan, w_min, w_max, &h) == RICK_OK) {
            rick_set_stream(h, st);
            const int bpsm[3] = {4, 16, 32};
            for (int k = 0; k < 3; ++k) {
                rick_set_prep_blocks(h, bpsm[k]);
                const double ms = time_batch(h, st, e0, e1, vis, u, v, w, weights, chan_offsets, images, kReps);
                if (ms > 0.0 && ms < best) {
                    best = ms;
                    best_pb = bpsm[k];
                }
            }
            rick_destroy(h);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(images);
    if (!best_t) return RICK_ERR_CUDA;
    *tile_out = best_t;
    *plane_group_out = best_g;
    if (prep_blocks_out) *prep_blocks_out = best_pb;
    if (ms_out) *ms_out = best;
    if (cache && *cache) {
        FILE* f = fopen(cache, "a");
        if (f) {
            fprintf(f, "%s|%d %d %d %.4f\n", key, best_t, best_g, best_pb, best);
            fclose(f);
        }
    }
    return RICK_OK;
}

rick_status rick_set_plane_range(rick_handle h, int32_t k0, int32_t k1)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: the plane range is single-image");
    if (!(0 <= k0 && k0 < k1 && k1 <= h->p.nw))
        return fail(h, RICK_ERR_ARG, "plane range [%d, %d) not within [0, %d)", (int)k0, (int)k1, (int)h->p.nw);
    if (!h->chunks.empty())
        return fail(h, RICK_ERR_STATE, "set the plane range before rick_grid (after rick_reset)");
    h->cfg.plane_lo = k0;
    h->cfg.plane_hi = k1;
    return RICK_OK;
}

rick_status rick_set_weight_sum(rick_handle h, double sum_w)
{
    if (!h) return RICK_ERR_ARG;
    if (h->batch) return fail(h, RICK_ERR_STATE, "batched handle: weight sums are per channel");
    if (std::isnan(sum_w) || std::isinf(sum_w)) return fail(h, RICK_ERR_ARG, "sum_w must be finite");
    if (sum_w < 0.0) {
        h->sw_given = false;
        return RICK_OK;
    }
    if (!h->sw_dev) {
        RICK_CU(h, cudaMalloc((void**)&h->sw_dev, sizeof(double)));
        h->bytes_held += sizeof(double);
    }
    // the host value is kept in the handle: the copy is ordered on the stream
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    h->sw_host = sum_w;
    RICK_CU(h, cudaMemcpy(h->sw_dev, &h->sw_host, sizeof(double), cudaMemcpyHostToDevice));
    h->sw_given = true;
    return RICK_OK;
}

rick_status rick_debug_colstack(rick_handle h, int32_t skip_slot, int64_t wait_ns)
{
    if (!h) return RICK_ERR_ARG;
    if (skip_slot < -1) return fail(h, RICK_ERR_ARG, "skip_slot must be >= -1 (got %d)", (int)skip_slot);
    h->dbg_skip_slot1 = skip_slot + 1;
    h->dbg_wait_ns = wait_ns > 0 ? (unsigned long long)wait_ns : 0ull;
    return RICK_OK;
}

rick_status rick_get_stats(rick_handle h, rick_stats* out)
{
    if (!h || !out) return RICK_ERR_ARG;
    Counters c;
    RICK_CU(h, cudaStreamSynchronize(h->stream));
    RICK_CU(h, cudaMemcpy(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost));
    if (c.err) return fail(h, RICK_ERR_TIMEOUT, "a bounded wait of the column-stack kernel ran out (image invalid)");
    out->n_gridded = (int64_t)c.gridded;
    out->n_dropped = (int64_t)c.dropped;
    out->n_entries = (int64_t)c.entries;
    out->sum_weights = c.sum_w;
    out->plane_group = h->G;
    out->tile = h->cfg.T;
    out->workspace_bytes = (int64_t)h->bytes_held;
    return RICK_OK;
}

}  // extern "C"
