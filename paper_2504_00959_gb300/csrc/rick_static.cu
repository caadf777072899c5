// rick_static.cu -- gridding without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns the whole device heap (a fixed arena handed out by
// the application), or real-time pipelines that forbid allocation after
// start-up because it may block or fragment.  rick_grid_planes_static serves
// them: it grids measurements into planes the caller provides, and every
// byte of working memory it needs comes from one fixed array in the
// library's static device data.
//
// The array is kStaticScratchBytes (64 MiB).  The library is built without
// relocatable device code, so this file is a module of its own; under CUDA's
// default lazy module loading the module, and with it the array, is loaded
// on a device at the first cudaGetSymbolAddress there -- the function's
// first call on that device -- and stays until the process exits.  That
// first call must therefore come before a framework claims the rest of the
// heap, and before any stream capture.  All calls on a device share the same array and it keeps the last
// call's contents, so calls whose GPU work overlaps (on different streams or
// from different host threads) race; the caller must order them.  Anything
// that must start at zero is cleared at the start of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rick_internal.cuh"

namespace rick {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;

// The scratch.  In host code `g_static_scratch` names a host-side stand-in,
// not device memory: only the address from cudaGetSymbolAddress may be passed
// to kernels.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceState {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    // tap polynomials of the last kernel configuration used on this device
    bool have_coef = false;
    int kernel = -1, support = -1;
    double kparam = 0.0;
    float coef[kMaxSupport][kPolyTerms];
};

std::mutex g_mutex;
DeviceState g_state[kMaxDevices];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

void set_msg(char* err, size_t err_len, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
void set_msg(char* err, size_t err_len, const char* fmt, ...)
{
    if (!err || err_len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, err_len, fmt, ap);
    va_end(ap);
}

}  // namespace
}  // namespace rick

using namespace rick;

extern "C" rick_status rick_grid_planes_static(const rick_params* p, const float* vis, const float* u,
                                               const float* v, const float* w, const float* weights, int64_t nvis,
                                               float* planes, void* cuda_stream, char* err, size_t err_len)
{
    if (err && err_len) err[0] = 0;
    GridCfg c;
    double kparam = 0.0;
    char msg[256];
    rick_status s = validate_params(p, &c, &kparam, msg, sizeof(msg));
    if (s) {
        set_msg(err, err_len, "%s", msg);
        return s;
    }
    c.cstride = counter_stride((int64_t)c.nw * c.ntp, kStaticCounterWords);  // the fixed scratch's budget
    if (nvis < 0 || nvis > ((int64_t)1 << 30)) {
        set_msg(err, err_len, "nvis must be in [0, 2^30] (got %lld)", (long long)nvis);
        return RICK_ERR_ARG;
    }
    if (!planes || (nvis > 0 && (!vis || !u || !v || !w))) {
        set_msg(err, err_len, "planes, vis, u, v, w must not be NULL");
        return RICK_ERR_ARG;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // scratch layout: counters | coefficients | cursor (+1 word) | offsets | scan sums | density | entries
    const int64_t ntiles = (int64_t)c.nw * c.ntp;
    const int64_t cap = nvis * (c.S > 1 ? 4 : 1) * c.Sw;
    const size_t o_ctr = 0;
    const size_t o_coef = o_ctr + align256(sizeof(Counters));
    const size_t o_err = o_coef + align256(sizeof(float) * kMaxSupport * kPolyTerms);
    const size_t o_cursor = o_err + align256(sizeof(double) * kMaxSupport);
    const size_t cursor_words = (size_t)ntiles * c.cstride + 1;
    const size_t o_off = o_cursor + align256(cursor_words * sizeof(uint32_t));
    const size_t o_sums = o_off + align256((size_t)(ntiles + 1) * sizeof(uint32_t));
    const size_t o_dens = o_sums + align256(scan_block_sums_len(ntiles) * sizeof(uint32_t));
    const size_t dens_bytes = c.uniform ? (size_t)c.n * c.n * sizeof(uint32_t) : 0;
    const size_t o_ent = o_dens + align256(dens_bytes);
    const size_t need = o_ent + (size_t)cap * sizeof(float4);
    if (need > kStaticScratchBytes) {
        set_msg(err, err_len,
                "rick_grid_planes_static: needs %zu bytes of scratch, the static limit is %zu bytes "
                "(n=%d, nw=%d, tile=%d, %lld measurements)",
                need, kStaticScratchBytes, c.n, c.nw, c.T, (long long)nvis);
        return RICK_ERR_ARG;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_msg(err, err_len, "no usable current CUDA device");
        return RICK_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState& ds = g_state[dev];
    if (!ds.ready) {
        // once per device, with that device current
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            set_msg(err, err_len, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            return RICK_ERR_CUDA;
        }
        ds.scratch = static_cast<unsigned char*>(ptr);
        ds.ready = true;
    }
    unsigned char* base = ds.scratch;
    Counters* ctr = reinterpret_cast<Counters*>(base + o_ctr);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(base + o_cursor);
    uint32_t* off = reinterpret_cast<uint32_t*>(base + o_off);
    uint32_t* sums = reinterpret_cast<uint32_t*>(base + o_sums);
    uint32_t* density = c.uniform ? reinterpret_cast<uint32_t*>(base + o_dens) : nullptr;
    float4* ent = reinterpret_cast<float4*>(base + o_ent);

    cudaError_t e = cudaSuccess;
    if (!(ds.have_coef && ds.kernel == p->kernel && ds.support == p->support && ds.kparam == kparam)) {
        // first call for this kernel configuration: fit the tap polynomials
        // into the scratch and fetch them (one synchronisation of the stream)
        float* d_coef = reinterpret_cast<float*>(base + o_coef);
        double* d_err = reinterpret_cast<double*>(base + o_err);
        float coef[kMaxSupport * kPolyTerms];
        double ferr[kMaxSupport];
        e = launch_fit_taps(c, kparam, d_coef, d_err, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(coef, d_coef, sizeof(coef), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ferr, d_err, sizeof(ferr), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            set_msg(err, err_len, "kernel tap fit: %s", cudaGetErrorString(e));
            return RICK_ERR_CUDA;
        }
        double worst = 0.0;
        for (int t = 0; t < c.S; ++t) worst = ferr[t] > worst ? ferr[t] : worst;
        if (!(worst <= 2e-6)) {
            set_msg(err, err_len, "kernel too sharp for the degree-10 tap polynomials (error %.2e)", worst);
            return RICK_ERR_ARG;
        }
        for (int t = 0; t < kMaxSupport; ++t)
            for (int j = 0; j < kPolyTerms; ++j) ds.coef[t][j] = (t < c.S) ? coef[t * kPolyTerms + j] : 0.0f;
        ds.kernel = p->kernel;
        ds.support = p->support;
        ds.kparam = kparam;
        ds.have_coef = true;
    }
    memcpy(c.coef, ds.coef, sizeof(c.coef));
    set_tap_sum(c);

    const float2* vis2 = reinterpret_cast<const float2*>(vis);
    e = cudaMemsetAsync(ctr, 0, sizeof(Counters), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)ntiles * c.cstride * sizeof(uint32_t), stream);
    if (e == cudaSuccess && density) e = cudaMemsetAsync(density, 0, dens_bytes, stream);
    if (e == cudaSuccess && density) e = launch_density(c, u, v, w, weights, vis2, nvis, density, stream);
    if (e == cudaSuccess) e = launch_count(c, u, v, w, weights, vis2, nvis, cursor, stream);
    if (e == cudaSuccess) e = launch_scan(cursor, ntiles, c.cstride, off, cursor, sums, stream);
    if (e == cudaSuccess) e = launch_scatter(c, u, v, w, weights, vis2, nvis, density, cursor, ent, ctr, nullptr, stream);
    if (e == cudaSuccess) {
        ChunkList cl{};
        cl.off[0] = off;
        cl.ent[0] = ent;
        cl.count = 1;
        // the scatter cursors are free again: they hold the gridder's heavy-tile list
        e = launch_grid(c, cl, 0, c.nw, false, false, cursor, cursor_words, reinterpret_cast<float2*>(planes),
                        stream);
    }
    if (e != cudaSuccess) {
        set_msg(err, err_len, "rick_grid_planes_static launch: %s", cudaGetErrorString(e));
        return RICK_ERR_CUDA;
    }
    return RICK_OK;
}
