// ppf_abi.cu -- the C ABI declared in include/ppf.h: plan validation, kernel
// selection, device tables, launches, the host-buffer pipeline and errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "../../include/ppf.h"
#include "ppf_bwd.cuh"
#include "ppf_bwd_unfused.cuh"
#include "ppf_fwd.cuh"
#include "ppf_internal.h"

namespace {

thread_local char g_msg[512] = "";

ppf_status fail(ppf_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

}  // namespace

ppf_status ppf::set_error(ppf_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

namespace {

ppf_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(PPF_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    return fail(PPF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr uint32_t kMagic = 0x50504631u;   // "PPF1"

int tap_bucket(int T) {
    if (T <= 1) return 1;
    if (T <= 2) return 2;
    if (T <= 4) return 4;
    if (T <= 8) return 8;
    if (T <= 16) return 16;
    return 64;
}

bool lookup(int C, int tm, int in, int out, ppf::FwdEntry* e) {
    switch (C) {
        case 32: return ppf::fwd_lookup_c32(tm, in, out, e);
        case 64: return ppf::fwd_lookup_c64(tm, in, out, e);
        case 128: return ppf::fwd_lookup_c128(tm, in, out, e);
        case 256: return ppf::fwd_lookup_c256(tm, in, out, e);
        case 512: return ppf::fwd_lookup_c512(tm, in, out, e);
        case 1024: return ppf::fwd_lookup_c1024(tm, in, out, e);
        case 2048: return ppf::fwd_lookup_c2048(tm, in, out, e);
        case 4096: return ppf::fwd_lookup_c4096(tm, in, out, e);
        case 384: return ppf::fwd_lookup_c384(tm, in, out, e);
        case 768: return ppf::fwd_lookup_c768(tm, in, out, e);
        case 1536: return ppf::fwd_lookup_c1536(tm, in, out, e);
        case 3072: return ppf::fwd_lookup_c3072(tm, in, out, e);
        default: return false;
    }
}

bool lookup_fir(int C, int tm, int in, ppf::FwdEntry* e) {
    switch (C) {
        case 32: return ppf::fir_lookup_c32(tm, in, e);
        case 64: return ppf::fir_lookup_c64(tm, in, e);
        case 128: return ppf::fir_lookup_c128(tm, in, e);
        case 256: return ppf::fir_lookup_c256(tm, in, e);
        case 512: return ppf::fir_lookup_c512(tm, in, e);
        case 1024: return ppf::fir_lookup_c1024(tm, in, e);
        case 2048: return ppf::fir_lookup_c2048(tm, in, e);
        case 4096: return ppf::fir_lookup_c4096(tm, in, e);
        case 384: return ppf::fir_lookup_c384(tm, in, e);
        case 768: return ppf::fir_lookup_c768(tm, in, e);
        case 1536: return ppf::fir_lookup_c1536(tm, in, e);
        case 3072: return ppf::fir_lookup_c3072(tm, in, e);
        default: return false;
    }
}

bool lookup_idft(int C, ppf::IdftEntry* e) {
    switch (C) {
#define PPF_ID(CC) case CC: return ppf::idft_lookup_c##CC(e);
        PPF_ID(32) PPF_ID(64) PPF_ID(128) PPF_ID(256) PPF_ID(512) PPF_ID(1024) PPF_ID(2048) PPF_ID(4096)
        PPF_ID(384) PPF_ID(768) PPF_ID(1536) PPF_ID(3072)
#undef PPF_ID
        default: return false;
    }
}

bool twiddles(int C, std::vector<float>& pairs) {
    int n = 0;
    switch (C) {
#define PPF_TW(CC) case CC: n = ppf::fwd_twiddle_count_c##CC(); pairs.assign(2 * n, 0.f); ppf::fwd_twiddles_c##CC(pairs.data()); return true;
        PPF_TW(32) PPF_TW(64) PPF_TW(128) PPF_TW(256) PPF_TW(512) PPF_TW(1024) PPF_TW(2048) PPF_TW(4096)
        PPF_TW(384) PPF_TW(768) PPF_TW(1536) PPF_TW(3072)
#undef PPF_TW
        default: return false;
    }
}

int bytes_in(ppf_in_t t) { return t == PPF_IN_CI8 ? 2 : t == PPF_IN_CI16 ? 4 : 8; }
int bytes_out(ppf_out_t t) { return t == PPF_OUT_CF32 ? 8 : 4; }

}  // namespace

// Host pipeline state of ppf_execute_host (allocated on first use).
// Three streams, one per engine: host->device copies, kernels,
// device->host copies, so at most one copy per direction is in flight (two
// concurrent copies in one direction share the host link no faster) and
// each engine works through its chunks in order.  kDepth staging slots;
// events order a slot's reuse after its last reader.
struct HostPipe {
    static constexpr int kDepth = 3;
    long long chunk = 0;                 // output spectra per chunk
    cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
    void* d_in[kDepth] = {};
    void* d_out[kDepth] = {};
    cudaEvent_t ev_in[kDepth] = {};      // slot's input landed
    cudaEvent_t ev_cmp[kDepth] = {};     // slot's kernel done (input free, output ready)
    cudaEvent_t ev_out[kDepth] = {};     // slot's output copied out (output free)
    cudaEvent_t start = nullptr;
};

struct ppf_plan_s {
    uint32_t magic;
    int C, T, TM, device, grid, sms, occupancy;
    ppf_in_t in;
    ppf_out_t out;
    float* d_taps;        // TM*C floats, rows >= T zero
    float2* d_tw;         // twiddle tables
    int* d_err;           // device status word written by bounded waits
    int debug_flags;      // testing aid: ppf::FwdFlags passed to the kernel
    ppf::FwdEntry fwd;
    HostPipe* pipe;
    bool has_bwd;         // adjoint kernel available for this shape
    ppf::BwdEntry bwd;
    int bwd_occupancy;
    float* d_partials;    // tap-gradient partial sums, one row of TM*C per CTA (or per part)
    long long partials_ctas;
    ppf::IdftEntry idft;  // unfused adjoint: inverse DFT pass
    int idft_occupancy;
    float2* d_gy;         // unfused adjoint: g_y scratch
    size_t gy_bytes;
    bool has_fir;         // FIR-only ablation kernel available for this shape
    ppf::FwdEntry fir;
    int fir_grid;
    ppf_plan_s* fft_sub;  // DFT-only ablation: a T=1, h=1, complex FP32 input plan (made on first use)
};

// Registry of live plans: a handle is checked against it before it is
// dereferenced, so a destroyed or foreign handle is rejected, not used.
static std::mutex g_plans_mu;
static std::unordered_set<const void*> g_plans;

static bool valid_plan(ppf_plan_t p) {
    if (p == nullptr) return false;
    std::lock_guard<std::mutex> lk(g_plans_mu);
    return g_plans.count(p) != 0 && p->magic == kMagic;
}
static void register_plan(ppf_plan_t p) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plans.insert(p);
}
static void unregister_plan(ppf_plan_t p) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plans.erase(p);
}

extern "C" const char* ppf_status_string(ppf_status s) {
    switch (s) {
        case PPF_OK: return "PPF_OK";
        case PPF_ERR_INVALID_ARG: return "PPF_ERR_INVALID_ARG";
        case PPF_ERR_UNSUPPORTED: return "PPF_ERR_UNSUPPORTED";
        case PPF_ERR_ALIGNMENT: return "PPF_ERR_ALIGNMENT";
        case PPF_ERR_CUDA: return "PPF_ERR_CUDA";
        case PPF_ERR_DEVICE_TIMEOUT: return "PPF_ERR_DEVICE_TIMEOUT";
        case PPF_ERR_OUT_OF_MEMORY: return "PPF_ERR_OUT_OF_MEMORY";
        default: return "PPF_ERR_UNKNOWN";
    }
}

extern "C" const char* ppf_last_error_message(void) { return g_msg; }

extern "C" ppf_status ppf_plan(ppf_plan_t* out, int C, int T, const float* coeffs_host,
                               ppf_in_t in_dtype, ppf_out_t out_dtype) {
    if (out == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_plan: out is NULL");
    *out = nullptr;
    if (coeffs_host == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_plan: coefficients are NULL");
    if (C < 1 || T < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_plan: C=%d, T=%d must be >= 1", C, T);
    const bool c3 = (C == 384 || C == 768 || C == 1536 || C == 3072);
    if (!c3 && ((C & (C - 1)) != 0 || C < PPF_MIN_CHANNELS || C > PPF_MAX_CHANNELS))
        return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: C=%d is neither a power of two in [%d, %d] nor 3*2^k in [384, 3072]",
                    C, PPF_MIN_CHANNELS, PPF_MAX_CHANNELS);
    if (T > PPF_MAX_TAPS) return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: T=%d > %d", T, PPF_MAX_TAPS);
    if (in_dtype < PPF_IN_CI8 || in_dtype > PPF_IN_CF32)
        return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: unknown input type %d", (int)in_dtype);
    if (out_dtype < PPF_OUT_CF32 || out_dtype > PPF_OUT_CF16)
        return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: unknown output type %d", (int)out_dtype);

    const int tm = tap_bucket(T);
    ppf::FwdEntry e{};
    if (!lookup(C, tm, (int)in_dtype, (int)out_dtype, &e))
        return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: no kernel for C=%d T=%d", C, T);

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_plan: cudaGetDevice");
    int sms = 0;
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_plan: SM count");
    ce = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_plan: shared memory attribute");
    int occ = 0, grid_ctas = 0;
    if (e.cluster > 0) {
        // persistent grid: as many whole clusters as can be resident at once
        int clusters = 0;
        ce = ppf::max_active_clusters(e, sms, &clusters);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_plan: cluster occupancy");
        if (clusters < 1) return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: a cluster of the kernel does not fit");
        grid_ctas = clusters * e.cluster;
        occ = (grid_ctas + sms - 1) / sms;   // CTAs per SM (reported)
    } else {
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn, e.threads, e.smem);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_plan: occupancy");
        if (occ < 1) return fail(PPF_ERR_UNSUPPORTED, "ppf_plan: kernel does not fit on an SM");
        grid_ctas = sms * occ;
    }

    // Device tables: taps padded to the bucket with zero rows (and 4 more zero
    // rows for the largest bucket: the long-tap kernel loads taps 4 ahead), twiddles.
    std::vector<float> taps((size_t)(tm == PPF_MAX_TAPS ? tm + 4 : tm) * C, 0.f);
    std::memcpy(taps.data(), coeffs_host, sizeof(float) * (size_t)C * T);
    std::vector<float> tw;
    twiddles(C, tw);

    ppf_plan_s* p = new (std::nothrow) ppf_plan_s{};
    if (p == nullptr) return fail(PPF_ERR_OUT_OF_MEMORY, "ppf_plan: host allocation");
    p->magic = kMagic;
    p->C = C; p->T = T; p->TM = tm; p->device = dev; p->sms = sms; p->occupancy = occ;
    p->grid = grid_ctas;
    p->in = in_dtype; p->out = out_dtype; p->fwd = e;
    if (ppf::bwd_lookup(C, tm, (int)in_dtype, &p->bwd)) {
        ce = cudaFuncSetAttribute(p->bwd.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->bwd.smem);
        if (ce == cudaSuccess)
            ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->bwd_occupancy, p->bwd.fn, p->bwd.threads, p->bwd.smem);
        if (ce != cudaSuccess) {
            delete p;
            return cuda_fail(ce, "ppf_plan: backward kernel attributes");
        }
        p->has_bwd = p->bwd_occupancy > 0;
    }
    if (lookup_idft(C, &p->idft)) {
        ce = cudaFuncSetAttribute(p->idft.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->idft.smem);
        if (ce == cudaSuccess)
            ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->idft_occupancy, p->idft.fn, p->idft.threads,
                                                               p->idft.smem);
        if (ce != cudaSuccess) {
            delete p;
            return cuda_fail(ce, "ppf_plan: inverse-DFT kernel attributes");
        }
    }
    if (lookup_fir(C, tm, (int)in_dtype, &p->fir)) {
        int focc = 0;
        ce = cudaFuncSetAttribute(p->fir.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->fir.smem);
        if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&focc, p->fir.fn, p->fir.threads, p->fir.smem);
        if (ce != cudaSuccess) {
            delete p;
            return cuda_fail(ce, "ppf_plan: FIR-only kernel attributes");
        }
        p->has_fir = focc > 0;
        p->fir_grid = sms * focc;
    }
    register_plan(p);
    ce = cudaMalloc(&p->d_taps, taps.size() * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_tw, tw.size() * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_err, 16);
    if (ce == cudaSuccess) ce = cudaMemset(p->d_err, 0, 16);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_taps, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        ppf_status s = cuda_fail(ce, "ppf_plan: device tables");
        ppf_destroy(p);
        return s;
    }
    *out = p;
    return PPF_OK;
}

cudaError_t ppf::max_active_clusters(const FwdEntry& e, int sms, int* clusters) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = e.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(e.cluster * sms, 1, 1);
    cfg.blockDim = dim3(e.threads, 1, 1);
    cfg.dynamicSmemBytes = e.smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    *clusters = 0;
    return cudaOccupancyMaxActiveClusters(clusters, e.fn, &cfg);
}

// Work units (CTAs, or clusters of CTAs) of one launch: one wave of resident
// units sharing the batches of all streams equally, at most one per batch.
static long long work_units(long long resident, long long n_streams, long long batches_per_stream) {
    const long long total = n_streams * batches_per_stream;
    return std::max<long long>(1, std::min<long long>(resident, total));
}

static ppf_status launch_fwd(ppf_plan_t p, const void* in_dev, long long in_stride, void* out_dev,
                             long long out_stride, long long n, long long n_streams, cudaStream_t st) {
    ppf::FwdArgs a;
    a.in = in_dev;
    a.out = out_dev;
    a.in_stride = in_stride;
    a.out_stride = out_stride;
    a.taps = p->d_taps;
    a.tw = p->d_tw;
    a.err = p->d_err;
    a.n_spectra = n;
    a.T = p->T;
    a.flags = p->debug_flags;
    const long long nb = (n + p->fwd.batch - 1) / p->fwd.batch;
    const int unit = p->fwd.cluster > 0 ? p->fwd.cluster : 1;      // CTAs per work unit
    a.n_streams = n_streams;
    long long grid;
    if ((p->fwd.variant & 4) && p->fwd.cluster == 0) {
        // carry kernel: the same number of CTAs on every stream, one wave if
        // the streams allow it (at least one CTA, at most one per batch)
        const long long cps = std::max<long long>(1, std::min<long long>(p->grid / n_streams, nb));
        grid = cps * n_streams;
        if (grid > 0x7fffffffll) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: too many streams");
    } else {
        grid = work_units(p->grid / unit, n_streams, nb) * unit;
    }
    cudaError_t ce = p->fwd.launch(a, (int)grid, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_execute: launch");
    return PPF_OK;
}

static bool overlaps(const void* a, unsigned long long na, const void* b, unsigned long long nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

extern "C" ppf_status ppf_execute_batched(ppf_plan_t p, const void* in_dev, long long in_stride, void* out_dev,
                                          long long out_stride, long long n_spectra, long long n_streams,
                                          ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: invalid plan");
    if (in_dev == nullptr || out_dev == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: NULL buffer");
    if (n_spectra < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: n_spectra=%lld < 1", n_spectra);
    if (n_streams < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: n_streams=%lld < 1", n_streams);
    const long long in_len = (long long)p->C * (n_spectra + p->T - 1), out_len = (long long)p->C * n_spectra;
    if (n_streams > 1 && (in_stride < in_len || out_stride < out_len))
        return fail(PPF_ERR_INVALID_ARG, "ppf_execute: stream strides shorter than one stream");
    const int bi = bytes_in(p->in), bo = bytes_out(p->out);
    if ((reinterpret_cast<uintptr_t>(in_dev) & 15) || (reinterpret_cast<uintptr_t>(out_dev) & 15) ||
        (n_streams > 1 && (((in_stride * bi) & 15) || ((out_stride * bo) & 15))))
        return fail(PPF_ERR_ALIGNMENT, "ppf_execute: buffers and stream strides must be 16-byte aligned");
    const unsigned long long in_bytes = (unsigned long long)((n_streams - 1) * in_stride + in_len) * bi;
    const unsigned long long out_bytes = (unsigned long long)((n_streams - 1) * out_stride + out_len) * bo;
    if (overlaps(in_dev, in_bytes, out_dev, out_bytes))
        return fail(PPF_ERR_INVALID_ARG, "ppf_execute: input and output overlap");
    return launch_fwd(p, in_dev, in_stride, out_dev, out_stride, n_spectra, n_streams,
                      reinterpret_cast<cudaStream_t>(stream));
}

extern "C" ppf_status ppf_execute(ppf_plan_t p, const void* in_dev, void* out_dev, long long n_spectra,
                                  ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_execute: invalid plan");
    return ppf_execute_batched(p, in_dev, 0, out_dev, 0, n_spectra, 1, stream);
}

// The unfused adjoint: inverse DFT of G into the plan's g_y scratch, then
// the grad_x pass and the grad_h partial sums + fixed-order reduction.
static ppf_status backward_unfused(ppf_plan_t p, const void* grad_out_dev, const void* in_dev, void* grad_in_dev,
                                   float* grad_taps_dev, long long n_spectra, long long n_streams, cudaStream_t st) {
    const int C = p->C, T = p->T, TM = p->TM;
    if (p->idft.fn == nullptr || p->idft_occupancy < 1)
        return fail(PPF_ERR_UNSUPPORTED, "ppf_backward: no inverse-DFT kernel for C=%d", C);
    const long long n_raw = n_spectra + T - 1;
    const size_t gy_bytes = (size_t)n_streams * n_spectra * C * 8;
    cudaError_t ce;
    if (gy_bytes > p->gy_bytes) {   // g_y scratch, grown when a call needs more
        if (p->d_gy) cudaFree(p->d_gy);
        p->d_gy = nullptr;
        p->gy_bytes = 0;
        ce = cudaMalloc(&p->d_gy, gy_bytes);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: g_y scratch");
        p->gy_bytes = gy_bytes;
    }
    ppf::IdftArgs ia;
    ia.gY = static_cast<const float2*>(grad_out_dev);
    ia.gy = p->d_gy;
    ia.tw = p->d_tw;
    ia.n_spectra = n_spectra;
    ia.gY_stride = n_spectra * C;
    ia.n_streams = n_streams;
    const long long idft_grid = work_units((long long)p->sms * p->idft_occupancy, n_streams,
                                           (n_spectra + p->idft.batch - 1) / p->idft.batch);
    ce = p->idft.launch(ia, (int)idft_grid, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: inverse DFT launch");
    if (grad_in_dev != nullptr) {
        ppf::AdjFirArgs fa;
        fa.gy = p->d_gy;
        fa.taps = p->d_taps;
        fa.gx = static_cast<float2*>(grad_in_dev);
        fa.n_spectra = n_spectra;
        fa.n_streams = n_streams;
        fa.gx_stride = n_raw * C;
        fa.C = C;
        fa.T = T;
        const long long tiles = n_streams * ((n_raw + ppf::kAdjL - 1) / ppf::kAdjL);
        const long long pair_blocks = (C / 2 + 127) / 128;
        const long long gx_grid = std::min<long long>(tiles, std::max<long long>(1, 16LL * p->sms / pair_blocks));
        ce = ppf::bwd_gradx(fa, (int)gx_grid, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: grad_in launch");
    }
    if (grad_taps_dev != nullptr) {
        // parts of the rows of all streams: about 8 CTAs per SM in all, at
        // least 64 rows per part, partial sums capped at 2^25 floats
        const long long blocks = ((C / 2 + 127) / 128) * (long long)ppf::bwd_gradh_tap_blocks(T);
        long long parts = std::max<long long>(1, (8LL * p->sms + blocks - 1) / blocks);
        parts = std::min<long long>(parts, std::max<long long>(1, n_streams * n_spectra / 64));
        parts = std::min<long long>(parts, std::max<long long>(1, (1LL << 25) / ((long long)TM * C)));
        if (parts > p->partials_ctas) {
            if (p->d_partials) cudaFree(p->d_partials);
            p->d_partials = nullptr;
            p->partials_ctas = 0;
            ce = cudaMalloc(&p->d_partials, sizeof(float) * (size_t)parts * TM * C);
            if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: partial sums");
            p->partials_ctas = parts;
        }
        ppf::AdjCorrArgs ca;
        ca.gy = p->d_gy;
        ca.x = in_dev;
        ca.partials = p->d_partials;
        ca.n_spectra = n_spectra;
        ca.n_streams = n_streams;
        ca.x_stride = n_raw * C;
        ca.C = C;
        ca.T = T;
        ca.TM = TM;
        ca.n_parts = (int)parts;
        ce = ppf::bwd_gradh((int)p->in, ca, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: grad_taps launch");
        ce = ppf::bwd_reduce(p->d_partials, (int)parts, T, TM, C, p->d_err, grad_taps_dev, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: tap-gradient reduction");
    }
    return PPF_OK;
}

extern "C" ppf_status ppf_backward(ppf_plan_t p, const void* grad_out_dev, const void* in_dev, void* grad_in_dev,
                                   float* grad_taps_dev, long long n_spectra, long long n_streams,
                                   ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_backward: invalid plan");
    if (grad_out_dev == nullptr || in_dev == nullptr || (grad_in_dev == nullptr && grad_taps_dev == nullptr))
        return fail(PPF_ERR_INVALID_ARG, "ppf_backward: NULL buffer");
    if (n_spectra < 1 || n_streams < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_backward: empty problem");
    const uintptr_t al = reinterpret_cast<uintptr_t>(grad_out_dev) | reinterpret_cast<uintptr_t>(in_dev) |
                         reinterpret_cast<uintptr_t>(grad_in_dev) | reinterpret_cast<uintptr_t>(grad_taps_dev);
    if (al & 15) return fail(PPF_ERR_ALIGNMENT, "ppf_backward: buffers must be 16-byte aligned");
    const int C = p->C, T = p->T, TM = p->TM;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n_raw = n_spectra + T - 1;
    const long long in_len = (long long)C * n_raw, out_len = (long long)C * n_spectra;
    if (grad_in_dev && overlaps(grad_in_dev, (unsigned long long)(n_streams * in_len * 8), in_dev,
                                (unsigned long long)(n_streams * in_len * bytes_in(p->in))))
        return fail(PPF_ERR_INVALID_ARG, "ppf_backward: grad_in overlaps the input");
    if (grad_in_dev && overlaps(grad_in_dev, (unsigned long long)(n_streams * in_len * 8), grad_out_dev,
                                (unsigned long long)(n_streams * out_len * 8)))
        return fail(PPF_ERR_INVALID_ARG, "ppf_backward: grad_in overlaps grad_out");
    if (!p->has_bwd || (p->debug_flags & PPF_DEBUG_UNFUSED_ADJOINT))
        return backward_unfused(p, grad_out_dev, in_dev, grad_in_dev, grad_taps_dev, n_spectra, n_streams, st);
    const long long nb = (n_raw + p->bwd.batch - 1) / p->bwd.batch;
    // one wave of resident CTAs sharing the batches of all streams equally
    const long long grid = work_units((long long)p->sms * p->bwd_occupancy, n_streams, nb);
    if (grid > p->partials_ctas) {   // scratch for the per-CTA tap-gradient partial sums
        if (p->d_partials) cudaFree(p->d_partials);
        p->d_partials = nullptr;
        p->partials_ctas = 0;
        cudaError_t ce = cudaMalloc(&p->d_partials, sizeof(float) * (size_t)grid * TM * C);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: partial sums");
        p->partials_ctas = grid;
    }
    ppf::BwdArgs a;
    a.gY = static_cast<const float2*>(grad_out_dev);
    a.x = in_dev;
    a.taps = p->d_taps;
    a.tw = p->d_tw;
    a.gx = static_cast<float2*>(grad_in_dev);
    a.partials = p->d_partials;
    a.err = p->d_err;
    a.n_spectra = n_spectra;
    a.gY_stride = out_len;
    a.x_stride = in_len;
    a.n_streams = n_streams;
    a.T = T;
    a.flags = p->debug_flags;
    cudaError_t ce = p->bwd.launch(a, (int)grid, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: launch");
    if (grad_taps_dev != nullptr) {
        ce = ppf::bwd_reduce(p->d_partials, (int)grid, T, TM, C, p->d_err, grad_taps_dev, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward: tap-gradient reduction");
    }
    return PPF_OK;
}

static void free_pipe(HostPipe* hp) {
    if (hp == nullptr) return;
    for (cudaStream_t st : {hp->s_in, hp->s_cmp, hp->s_out})
        if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (int i = 0; i < HostPipe::kDepth; ++i) {
        if (hp->d_in[i]) cudaFree(hp->d_in[i]);
        if (hp->d_out[i]) cudaFree(hp->d_out[i]);
        for (cudaEvent_t ev : {hp->ev_in[i], hp->ev_cmp[i], hp->ev_out[i]})
            if (ev) cudaEventDestroy(ev);
    }
    if (hp->start) cudaEventDestroy(hp->start);
    delete hp;
}

extern "C" ppf_status ppf_execute_host(ppf_plan_t p, const void* in_host, void* out_host, long long n_spectra,
                                       ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_execute_host: invalid plan");
    if (in_host == nullptr || out_host == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_execute_host: NULL buffer");
    if (n_spectra < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_execute_host: n_spectra=%lld < 1", n_spectra);
    cudaError_t ce;
    const int C = p->C, T = p->T, bi = bytes_in(p->in), bo = bytes_out(p->out);
    if (p->pipe == nullptr) {
        HostPipe* hp = new (std::nothrow) HostPipe{};
        if (hp == nullptr) return fail(PPF_ERR_OUT_OF_MEMORY, "ppf_execute_host: host allocation");
        // ~64 MiB of output per chunk, a whole number of CTA batches
        long long ch = (64ll << 20) / ((long long)C * bo);
        ch = ch / p->fwd.batch * p->fwd.batch;
        if (ch < p->fwd.batch) ch = p->fwd.batch;
        hp->chunk = ch;
        const unsigned evf = cudaEventDisableTiming;
        ce = cudaEventCreateWithFlags(&hp->start, evf);
        for (cudaStream_t* st : {&hp->s_in, &hp->s_cmp, &hp->s_out})
            if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
        for (int i = 0; i < HostPipe::kDepth && ce == cudaSuccess; ++i) {
            ce = cudaMalloc(&hp->d_in[i], (size_t)C * (ch + T - 1) * bi);
            if (ce == cudaSuccess) ce = cudaMalloc(&hp->d_out[i], (size_t)C * ch * bo);
            for (cudaEvent_t* ev : {&hp->ev_in[i], &hp->ev_cmp[i], &hp->ev_out[i]})
                if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(ev, evf);
        }
        if (ce != cudaSuccess) {
            free_pipe(hp);
            return cuda_fail(ce, "ppf_execute_host: staging buffers");
        }
        p->pipe = hp;
    }
    HostPipe* hp = p->pipe;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    ce = cudaEventRecord(hp->start, user);
    for (cudaStream_t st : {hp->s_in, hp->s_cmp, hp->s_out})
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, hp->start, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_execute_host: stream ordering");
    // chunk k in slot q = k % depth: H2D(k) on s_in after the kernel of chunk
    // k-depth has read slot q; the kernel on s_cmp after H2D(k) and after the
    // D2H of chunk k-depth has emptied output slot q; D2H(k) on s_out after
    // the kernel.  (Each wait binds to the event's latest record, i.e. the
    // one of chunk k-depth, or to none on the first use of a slot.)
    long long k = 0;
    for (long long s0 = 0; s0 < n_spectra; s0 += hp->chunk, ++k) {
        const int q = (int)(k % HostPipe::kDepth);
        const bool reuse = k >= HostPipe::kDepth;
        const long long n = (n_spectra - s0 < hp->chunk) ? n_spectra - s0 : hp->chunk;
        const char* src = static_cast<const char*>(in_host) + (size_t)s0 * C * bi;
        char* dst = static_cast<char*>(out_host) + (size_t)s0 * C * bo;
        if (reuse) ce = cudaStreamWaitEvent(hp->s_in, hp->ev_cmp[q], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(hp->d_in[q], src, (size_t)C * (n + T - 1) * bi, cudaMemcpyHostToDevice, hp->s_in);
        if (ce == cudaSuccess) ce = cudaEventRecord(hp->ev_in[q], hp->s_in);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(hp->s_cmp, hp->ev_in[q], 0);
        if (ce == cudaSuccess && reuse) ce = cudaStreamWaitEvent(hp->s_cmp, hp->ev_out[q], 0);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_execute_host: host->device copy");
        ppf_status s = launch_fwd(p, hp->d_in[q], 0, hp->d_out[q], 0, n, 1, hp->s_cmp);
        if (s != PPF_OK) return s;
        ce = cudaEventRecord(hp->ev_cmp[q], hp->s_cmp);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(hp->s_out, hp->ev_cmp[q], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(dst, hp->d_out[q], (size_t)C * n * bo, cudaMemcpyDeviceToHost, hp->s_out);
        if (ce == cudaSuccess) ce = cudaEventRecord(hp->ev_out[q], hp->s_out);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_execute_host: device->host copy");
    }
    for (cudaStream_t st : {hp->s_in, hp->s_cmp, hp->s_out}) {
        ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_execute_host: synchronise");
    }
    return PPF_OK;
}

extern "C" ppf_status ppf_destroy(ppf_plan_t p) {
    if (p == nullptr) return PPF_OK;
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_destroy: invalid plan");
    unregister_plan(p);
    if (p->fft_sub) ppf_destroy(p->fft_sub);
    free_pipe(p->pipe);
    if (p->d_taps) cudaFree(p->d_taps);
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->d_err) cudaFree(p->d_err);
    if (p->d_partials) cudaFree(p->d_partials);
    if (p->d_gy) cudaFree(p->d_gy);
    p->magic = 0;
    delete p;
    return PPF_OK;
}

extern "C" ppf_status ppf_plan_info(ppf_plan_t p, int info[8]) {
    if (!valid_plan(p) || info == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_plan_info: invalid argument");
    info[0] = p->fwd.threads;
    info[1] = p->fwd.batch;
    info[2] = p->grid;
    info[3] = p->fwd.smem;
    info[4] = p->TM;
    info[5] = p->fwd.stages;
    info[6] = p->fwd.variant;
    info[7] = p->occupancy;
    return PPF_OK;
}

extern "C" ppf_status ppf_check_device(ppf_plan_t p, ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_check_device: invalid plan");
    int v = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaMemcpyAsync(&v, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_check_device");
    if (v != 0) {
        ce = cudaMemsetAsync(p->d_err, 0, sizeof(int), st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_check_device: reset");
        return fail(PPF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait gave up; the launch returned early");
    }
    return PPF_OK;
}

extern "C" ppf_status ppf_set_debug_flags(ppf_plan_t p, int flags) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_set_debug_flags: invalid plan");
    if (flags & ~(PPF_DEBUG_INJECT_TIMEOUT | PPF_DEBUG_UNFUSED_ADJOINT))
        return fail(PPF_ERR_INVALID_ARG, "ppf_set_debug_flags: unknown flag");
    p->debug_flags = flags;
    return PPF_OK;
}

extern "C" ppf_status ppf_update_taps(ppf_plan_t p, const float* taps_dev, ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_update_taps: invalid plan");
    if (taps_dev == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_update_taps: NULL taps");
    cudaError_t ce = cudaMemcpyAsync(p->d_taps, taps_dev, sizeof(float) * (size_t)p->C * p->T,
                                     cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_update_taps");
    return PPF_OK;
}

// ---------------------------------------------------------------------------
// Backward pass without any allocation.
//
// Some callers cannot allocate device memory where they run the PFB: a
// real-time pipeline stage with a fixed device-memory budget set at start-up,
// or a loop where a cudaMalloc (which may synchronise the device or fail
// under memory pressure) is not allowed.  For them the tap-gradient partial
// sums of ppf_backward live in this fixed file-scope array instead of plan
// memory.  Every GPU that loads the library holds the array until the process
// exits.
// ---------------------------------------------------------------------------
#define PPF_NOALLOC_PARTIALS_FLOATS (1 << 19)   // 2 MiB of partial sums

static __device__ __align__(256) float g_noalloc_partials[PPF_NOALLOC_PARTIALS_FLOATS];

// Device address of g_noalloc_partials for each device, looked up once with
// that device current (the host-side name is only a stand-in).
static std::mutex g_noalloc_mu;
static std::vector<float*> g_noalloc_ptr;

static ppf_status noalloc_scratch(int dev, float** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
    if (g_noalloc_ptr[dev] == nullptr) {
        int cur = -1;
        cudaError_t ce = cudaGetDevice(&cur);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward_noalloc: cudaGetDevice");
        if (cur != dev) return fail(PPF_ERR_INVALID_ARG, "ppf_backward_noalloc: the plan's device is not current");
        float* ptr = nullptr;
        ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_partials);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return PPF_OK;
}

extern "C" ppf_status ppf_backward_noalloc(ppf_plan_t p, const void* grad_out_dev, const void* in_dev,
                                           void* grad_in_dev, float* grad_taps_dev, long long n_spectra,
                                           long long n_streams, ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_backward_noalloc: invalid plan");
    if (!p->has_bwd)
        return fail(PPF_ERR_UNSUPPORTED, "ppf_backward_noalloc: needs C in [64, 512] with T <= 16 (T <= 8 at C = 512)");
    if (grad_out_dev == nullptr || in_dev == nullptr || (grad_in_dev == nullptr && grad_taps_dev == nullptr))
        return fail(PPF_ERR_INVALID_ARG, "ppf_backward_noalloc: NULL buffer");
    if (n_spectra < 1 || n_streams < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_backward_noalloc: empty problem");
    const uintptr_t al = reinterpret_cast<uintptr_t>(grad_out_dev) | reinterpret_cast<uintptr_t>(in_dev) |
                         reinterpret_cast<uintptr_t>(grad_in_dev) | reinterpret_cast<uintptr_t>(grad_taps_dev);
    if (al & 15) return fail(PPF_ERR_ALIGNMENT, "ppf_backward_noalloc: buffers must be 16-byte aligned");
    const int C = p->C, T = p->T, TM = p->TM;
    const long long n_raw = n_spectra + T - 1;
    const long long in_len = (long long)C * n_raw, out_len = (long long)C * n_spectra;
    if (grad_in_dev && overlaps(grad_in_dev, (unsigned long long)(n_streams * in_len * 8), in_dev,
                                (unsigned long long)(n_streams * in_len * bytes_in(p->in))))
        return fail(PPF_ERR_INVALID_ARG, "ppf_backward_noalloc: grad_in overlaps the input");
    // one row of TM*C partial sums per CTA; fewer CTAs per stream if the array is short
    const long long row = (long long)TM * C;
    const long long max_ctas = PPF_NOALLOC_PARTIALS_FLOATS / row;
    float* partials = nullptr;
    ppf_status st = noalloc_scratch(p->device, &partials);
    if (st != PPF_OK) return st;
    const long long nb = (n_raw + p->bwd.batch - 1) / p->bwd.batch;
    const long long grid = std::min<long long>(work_units((long long)p->sms * p->bwd_occupancy, n_streams, nb), max_ctas);
    ppf::BwdArgs a;
    a.gY = static_cast<const float2*>(grad_out_dev);
    a.x = in_dev;
    a.taps = p->d_taps;
    a.tw = p->d_tw;
    a.gx = static_cast<float2*>(grad_in_dev);
    a.partials = partials;    // every CTA overwrites its whole row: nothing needs clearing
    a.err = p->d_err;
    a.n_spectra = n_spectra;
    a.gY_stride = out_len;
    a.x_stride = in_len;
    a.n_streams = n_streams;
    a.T = T;
    a.flags = p->debug_flags;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = p->bwd.launch(a, (int)grid, cs);
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward_noalloc: launch");
    if (grad_taps_dev != nullptr) {
        ce = ppf::bwd_reduce(partials, (int)grid, T, TM, C, p->d_err, grad_taps_dev, cs);
        if (ce != cudaSuccess) return cuda_fail(ce, "ppf_backward_noalloc: tap-gradient reduction");
    }
    return PPF_OK;
}

// ---------------------------------------------------------------------------
// Unfused ablation: the FIR and the DFT as two separate launches with the
// filtered spectra in global memory between them (the paper's structure).
// ---------------------------------------------------------------------------
extern "C" ppf_status ppf_fir(ppf_plan_t p, const void* in_dev, void* y_dev, long long n_spectra,
                              ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_fir: invalid plan");
    if (!p->has_fir)
        return fail(PPF_ERR_UNSUPPORTED, "ppf_fir: needs C in {64, 128, 256, 512} (1024 for int8) and T <= 16");
    if (in_dev == nullptr || y_dev == nullptr) return fail(PPF_ERR_INVALID_ARG, "ppf_fir: NULL buffer");
    if (n_spectra < 1) return fail(PPF_ERR_INVALID_ARG, "ppf_fir: n_spectra=%lld < 1", n_spectra);
    if ((reinterpret_cast<uintptr_t>(in_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 15)
        return fail(PPF_ERR_ALIGNMENT, "ppf_fir: buffers must be 16-byte aligned");
    const unsigned long long in_bytes = (unsigned long long)p->C * (n_spectra + p->T - 1) * bytes_in(p->in);
    if (overlaps(in_dev, in_bytes, y_dev, (unsigned long long)p->C * n_spectra * 8))
        return fail(PPF_ERR_INVALID_ARG, "ppf_fir: input and output overlap");
    ppf::FwdArgs a;
    a.in = in_dev;
    a.out = y_dev;
    a.in_stride = 0;
    a.out_stride = 0;
    a.taps = p->d_taps;
    a.tw = p->d_tw;
    a.err = p->d_err;
    a.n_spectra = n_spectra;
    a.T = p->T;
    a.flags = p->debug_flags;
    const long long nb = (n_spectra + p->fir.batch - 1) / p->fir.batch;
    a.n_streams = 1;
    cudaError_t ce = p->fir.launch(a, (int)work_units(p->fir_grid, 1, nb), reinterpret_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return cuda_fail(ce, "ppf_fir: launch");
    return PPF_OK;
}

extern "C" ppf_status ppf_fft(ppf_plan_t p, const void* y_dev, void* out_dev, long long n_spectra,
                              ppf_stream_t stream) {
    if (!valid_plan(p)) return fail(PPF_ERR_INVALID_ARG, "ppf_fft: invalid plan");
    if (p->fft_sub == nullptr) {
        std::vector<float> ones((size_t)p->C, 1.0f);
        ppf_plan_t sub = nullptr;
        ppf_status st = ppf_plan(&sub, p->C, 1, ones.data(), PPF_IN_CF32, p->out);
        if (st != PPF_OK) return st;
        p->fft_sub = sub;
    }
    return ppf_execute(p->fft_sub, y_dev, out_dev, n_spectra, stream);
}
