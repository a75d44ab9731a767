// ppf_beams.cu -- many independent beams with uneven channel counts, taps and
// spectrum counts in ONE persistent launch.
//
// The plan cuts every beam into tiles (contiguous ranges of output batches of
// about `tile_samples` samples) and sorts the tiles largest first in two
// queues: beams with C >= 1024 ("wide" tiles) and beams with C <= 512
// ("narrow" tiles).  The grid is persistent: one CTA of 512 threads per SM.
// Each CTA first pulls wide tiles from a device counter and runs each with
// the whole CTA: at C = 1024 the body of the carry kernel (one channel pair
// per thread, the FIR halo carried in registers, warp-local DFT stages), at
// C >= 2048 the body of the generic kernel (raw rows and their halo staged
// through a TMA ring).  When the wide queue is empty, the CTA splits into two
// groups of 256 threads, each with half of the shared memory and its own
// named barrier, and each group pulls narrow tiles from the second counter
// and runs them independently with the generic body.
// Both counters are reset by one memset before the launch, so the pair can
// be captured in a CUDA graph.  The body of each tile is chosen by the beam's
// (C, tap bucket) class.  Complex int8 input, complex FP32 output: the
// multi-beam workload of the channeliser.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/ppf.h"
#include "ppf_fwd.cuh"
#include "ppf_internal.h"

// C = 512 tiles on the carry body of a half-CTA group measured 2 % slower on
// the C <= 512 beams of the 96-beam set than on fwd_range (and equal on the
// whole set), so they run fwd_range unless this is set.
#ifndef PPF_BEAMS_CARRY512
#define PPF_BEAMS_CARRY512 0
#endif

namespace ppf {

constexpr int kBeamThreads = 512;                 // one CTA per SM
constexpr int kNarrowThreads = 256;               // a group of a CTA running narrow tiles
constexpr int kBeamC[] = {64, 128, 256, 512, 1024, 2048, 4096};
constexpr int kBeamTM[] = {4, 8, 16};
constexpr int kNumC = 7, kNumTM = 3;
constexpr int kFirstWide = 4;                     // kBeamC[4] = 1024: wide from here on

struct BeamDesc {
    const void* in;          // C*(S+T-1) complex int8 samples
    void* out;               // S*C complex FP32 outputs
    const float* taps;       // TM*C floats (rows >= T zero)
    const float2* tw;        // twiddle tables of C
    long long n_spectra;
    int C, T, cls;           // cls = index of (C, TM) in the compiled class table
};

struct BeamTile {
    long long lo, hi;        // output batches [lo, hi) of the beam
    int beam;
};

struct BeamsArgs {
    const BeamDesc* beams;
    const BeamTile* tiles;       // wide tiles [0, n_wide), then narrow tiles
    unsigned long long* queue;   // [0]: next wide tile, [1]: next narrow tile
    int* err;
    long long n_wide, n_narrow;
    int flags;
};

template <int CI> constexpr int class_threads() { return CI >= kFirstWide ? kBeamThreads : kNarrowThreads; }
// C = 1024 (the whole CTA): the carry kernel's body, whose
// one-channel-pair-per-thread shape matches the group; the other classes
// run fwd_range
template <int CI, int TI>
constexpr bool class_carry() {
    constexpr int C = kBeamC[CI], TM = kBeamTM[TI];
    if constexpr ((C == 512 && PPF_BEAMS_CARRY512) || C == 1024) {
        using S = CarryShape<C, TM, IN_CI8>;
        return S::OK && S::NT == class_threads<CI>();
    } else {
        return false;
    }
}

template <int CI, int TI, class GRP>
__device__ __forceinline__ bool beam_tile(const BeamsArgs& a, const BeamDesc& d, const BeamTile& t,
                                          unsigned char* smem) {
    constexpr int C = kBeamC[CI], TM = kBeamTM[TI];
    FwdArgs fa;
    fa.in = d.in;
    fa.out = d.out;
    fa.in_stride = 0;
    fa.out_stride = 0;
    fa.n_streams = 1;
    fa.taps = d.taps;
    fa.tw = d.tw;
    fa.err = a.err;
    fa.n_spectra = d.n_spectra;
    fa.T = d.T;
    fa.flags = a.flags;
    if constexpr (class_carry<CI, TI>())
        return carry_range<C, TM, IN_CI8, OUT_CF32, false, GRP, true>(fa, d.in, d.out, t.lo, t.hi, smem);
    else
        return fwd_range<C, TM, IN_CI8, OUT_CF32, class_threads<CI>(), GRP>(fa, d.in, d.out, t.lo, t.hi, smem);
}

// run tile t with the body of class cls, among classes with C index in [CI, CEND)
template <int CI, int TI, int CEND, class GRP>
__device__ __forceinline__ bool beam_dispatch(int cls, const BeamsArgs& a, const BeamDesc& d, const BeamTile& t,
                                              unsigned char* smem) {
    if (cls == CI * kNumTM + TI) return beam_tile<CI, TI, GRP>(a, d, t, smem);
    if constexpr (TI + 1 < kNumTM) return beam_dispatch<CI, TI + 1, CEND, GRP>(cls, a, d, t, smem);
    else if constexpr (CI + 1 < CEND) return beam_dispatch<CI + 1, 0, CEND, GRP>(cls, a, d, t, smem);
    else return true;
}

template <int CI, int TI>
constexpr int class_smem_of() {
    if constexpr (class_carry<CI, TI>()) return CarryShape<kBeamC[CI], kBeamTM[TI], IN_CI8>::SMEM;
    else return FwdShape<kBeamC[CI], kBeamTM[TI], IN_CI8, class_threads<CI>()>::SMEM;
}
template <int CI, int TI, int CEND>
constexpr int class_smem_max() {
    constexpr int s = class_smem_of<CI, TI>();
    if constexpr (TI + 1 < kNumTM) return s > class_smem_max<CI, TI + 1, CEND>() ? s : class_smem_max<CI, TI + 1, CEND>();
    else if constexpr (CI + 1 < CEND) return s > class_smem_max<CI + 1, 0, CEND>() ? s : class_smem_max<CI + 1, 0, CEND>();
    else return s;
}
template <int CI, int TI>
constexpr int class_batch(int cls) {
    if (cls == CI * kNumTM + TI)
        return class_carry<CI, TI>() ? CarryShape<kBeamC[CI], kBeamTM[TI], IN_CI8>::B
                                     : FwdShape<kBeamC[CI], kBeamTM[TI], IN_CI8, class_threads<CI>()>::B;
    if constexpr (TI + 1 < kNumTM) return class_batch<CI, TI + 1>(cls);
    else if constexpr (CI + 1 < kNumC) return class_batch<CI + 1, 0>(cls);
    else return 0;
}
// shared memory of a narrow group (128-byte multiple) and of the CTA
constexpr int kNarrowSmem = (class_smem_max<0, 0, kFirstWide>() + 127) / 128 * 128;
constexpr int kWideSmem = class_smem_max<kFirstWide, 0, kNumC>();
constexpr int kBeamSmem = kWideSmem > 2 * kNarrowSmem ? kWideSmem : 2 * kNarrowSmem;

__global__ void __launch_bounds__(kBeamThreads, 1) pfb_beams_kernel(BeamsArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long s_tile[2];
    // wide tiles: the whole CTA
    for (;;) {
        if (threadIdx.x == 0) s_tile[0] = atomicAdd(&a.queue[0], 1ull);
        __syncthreads();
        const unsigned long long ti = s_tile[0];
        __syncthreads();
        if (ti >= (unsigned long long)a.n_wide) break;
        const BeamTile t = a.tiles[ti];
        const BeamDesc d = a.beams[t.beam];
        if (!beam_dispatch<kFirstWide, 0, kNumC, CtaGroup>(d.cls, a, d, t, smem)) return;
    }
    // narrow tiles: two independent groups, each with half of the shared memory
    using G = HalfGroup<kNarrowThreads>;
    const int g = threadIdx.x / kNarrowThreads;
    unsigned char* gsmem = smem + g * kNarrowSmem;
    for (;;) {
        if (G::tid() == 0) s_tile[g] = atomicAdd(&a.queue[1], 1ull);
        G::sync();
        const unsigned long long ti = s_tile[g];
        G::sync();
        if (ti >= (unsigned long long)a.n_narrow) return;
        const BeamTile t = a.tiles[a.n_wide + ti];
        const BeamDesc d = a.beams[t.beam];
        if (!beam_dispatch<0, 0, kFirstWide, G>(d.cls, a, d, t, gsmem)) return;
    }
}

// twiddles of every supported C (host)
void fill_beam_twiddles(int C, std::vector<float2>& tw) {
    switch (C) {
#define PPF_BTW(CC) case CC: tw.assign(tw_total_float2s(CC) > 0 ? tw_total_float2s(CC) : 1, make_float2(0.f, 0.f)); fill_twiddles<CC>(tw.data()); break;
        PPF_BTW(64) PPF_BTW(128) PPF_BTW(256) PPF_BTW(512) PPF_BTW(1024) PPF_BTW(2048) PPF_BTW(4096)
#undef PPF_BTW
        default: tw.clear();
    }
}

}  // namespace ppf

namespace {

ppf_status bcuda(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return ppf::set_error(PPF_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    return ppf::set_error(PPF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr uint32_t kBeamsMagic = 0x50504642u;   // "PPFB"

int class_of(int C, int T) {
    int ci = -1, ti = -1;
    for (int i = 0; i < ppf::kNumC; ++i)
        if (ppf::kBeamC[i] == C) ci = i;
    for (int i = 0; i < ppf::kNumTM; ++i)
        if (T <= ppf::kBeamTM[i]) { ti = i; break; }
    return (ci < 0 || ti < 0) ? -1 : ci * ppf::kNumTM + ti;
}

}  // namespace

struct ppf_beams_s {
    uint32_t magic;
    int n_beams, sms, occupancy;
    long long tile_samples;
    std::vector<ppf::BeamDesc> host;       // descriptors (pointers bound by ppf_beams_bind)
    std::vector<int> tm;                   // tap bucket per beam
    ppf::BeamDesc* d_beams;
    ppf::BeamTile* d_tiles;                // wide tiles, then narrow tiles
    long long n_wide, n_narrow;
    unsigned long long* d_queue;
    int* d_err;
    float* d_taps;                         // all beams' taps, concatenated
    float2* d_tw;                          // twiddles of each distinct C, concatenated
    bool bound;
};

static std::mutex g_beams_mu;
static std::unordered_set<const void*> g_beams;

static bool valid_beams(ppf_beams_t b) {
    if (b == nullptr) return false;
    std::lock_guard<std::mutex> lk(g_beams_mu);
    return g_beams.count(b) != 0 && b->magic == kBeamsMagic;
}

// Cut every beam into tiles of about tile_samples samples (whole output
// batches of its class); wide tiles (C >= 2048) first, each queue sorted by
// work (samples x tap bucket) largest first.
static ppf_status build_tiles(ppf_beams_t b, long long tile_samples) {
    std::vector<ppf::BeamTile> tiles[2];
    std::vector<long long> weight[2];
    for (int i = 0; i < b->n_beams; ++i) {
        const ppf::BeamDesc& d = b->host[i];
        const int q = d.C >= ppf::kBeamC[ppf::kFirstWide] ? 0 : 1;
        const long long B = ppf::class_batch<0, 0>(d.cls);
        const long long nbt = (d.n_spectra + B - 1) / B;
        long long per = tile_samples / (B * d.C);
        if (per < 1) per = 1;
        for (long long lo = 0; lo < nbt; lo += per) {
            const long long hi = std::min(nbt, lo + per);
            tiles[q].push_back(ppf::BeamTile{lo, hi, i});
            weight[q].push_back((hi - lo) * B * d.C * (long long)b->tm[i]);
        }
    }
    std::vector<ppf::BeamTile> sorted;
    for (int q = 0; q < 2; ++q) {
        std::vector<size_t> order(tiles[q].size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return weight[q][x] > weight[q][y]; });
        for (size_t i : order) sorted.push_back(tiles[q][i]);
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    cudaError_t ce = cudaMalloc(&b->d_tiles, sizeof(ppf::BeamTile) * std::max<size_t>(1, sorted.size()));
    if (ce == cudaSuccess)
        ce = cudaMemcpy(b->d_tiles, sorted.data(), sizeof(ppf::BeamTile) * sorted.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams: tiles");
    b->n_wide = (long long)tiles[0].size();
    b->n_narrow = (long long)tiles[1].size();
    b->tile_samples = tile_samples;
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_destroy(ppf_beams_t b) {
    if (b == nullptr) return PPF_OK;
    if (!valid_beams(b)) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_destroy: invalid handle");
    {
        std::lock_guard<std::mutex> lk(g_beams_mu);
        g_beams.erase(b);
    }
    cudaFree(b->d_beams);
    cudaFree(b->d_tiles);
    cudaFree(b->d_queue);
    cudaFree(b->d_err);
    cudaFree(b->d_taps);
    cudaFree(b->d_tw);
    b->magic = 0;
    delete b;
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_plan(ppf_beams_t* out, int n_beams, const int* C, const int* T,
                                     const long long* n_spectra, const float* const* taps_host,
                                     ppf_in_t in_dtype, ppf_out_t out_dtype) {
    if (out == nullptr) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_plan: out is NULL");
    *out = nullptr;
    if (n_beams < 1 || C == nullptr || T == nullptr || n_spectra == nullptr || taps_host == nullptr)
        return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_plan: empty or NULL beam table");
    if (in_dtype != PPF_IN_CI8 || out_dtype != PPF_OUT_CF32)
        return ppf::set_error(PPF_ERR_UNSUPPORTED, "ppf_beams_plan: multi-beam launch takes complex int8 in, complex FP32 out");
    for (int i = 0; i < n_beams; ++i) {
        if (taps_host[i] == nullptr || n_spectra[i] < 1 || T[i] < 1)
            return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_plan: beam %d: bad taps, T or spectra", i);
        if (class_of(C[i], T[i]) < 0)
            return ppf::set_error(PPF_ERR_UNSUPPORTED, "ppf_beams_plan: beam %d: C=%d T=%d (needs C a power of two in [64, 4096], T <= 16)",
                         i, C[i], T[i]);
    }
    int dev = 0, sms = 0, occ = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(ppf::pfb_beams_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ppf::kBeamSmem);
    if (ce == cudaSuccess)
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf::pfb_beams_kernel, ppf::kBeamThreads, ppf::kBeamSmem);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_plan: device attributes");
    if (occ < 1) return ppf::set_error(PPF_ERR_UNSUPPORTED, "ppf_beams_plan: kernel does not fit on an SM");

    ppf_beams_s* b = new (std::nothrow) ppf_beams_s{};
    if (b == nullptr) return ppf::set_error(PPF_ERR_OUT_OF_MEMORY, "ppf_beams_plan: host allocation");
    b->magic = kBeamsMagic;
    b->n_beams = n_beams;
    b->sms = sms;
    b->occupancy = occ;
    b->host.resize(n_beams);
    b->tm.resize(n_beams);
    // taps (padded to the bucket) and twiddles (one table per distinct C)
    std::vector<float> taps;
    std::vector<long long> taps_off(n_beams);
    std::vector<float2> tw_all, tw;
    std::unordered_map<int, long long> tw_off;
    for (int i = 0; i < n_beams; ++i) {
        const int cls = class_of(C[i], T[i]);
        const int tmv = ppf::kBeamTM[cls % ppf::kNumTM];
        b->tm[i] = tmv;
        taps_off[i] = (long long)taps.size();
        taps.resize(taps.size() + (size_t)tmv * C[i], 0.f);
        std::memcpy(taps.data() + taps_off[i], taps_host[i], sizeof(float) * (size_t)C[i] * T[i]);
        if (!tw_off.count(C[i])) {
            ppf::fill_beam_twiddles(C[i], tw);
            tw_off[C[i]] = (long long)tw_all.size();
            tw_all.insert(tw_all.end(), tw.begin(), tw.end());
        }
        b->host[i] = ppf::BeamDesc{nullptr, nullptr, nullptr, nullptr, n_spectra[i], C[i], T[i], cls};
    }
    ce = cudaMalloc(&b->d_taps, sizeof(float) * taps.size());
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_tw, sizeof(float2) * std::max<size_t>(1, tw_all.size()));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_beams, sizeof(ppf::BeamDesc) * n_beams);
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_queue, 2 * sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_err, 16);
    if (ce == cudaSuccess) ce = cudaMemset(b->d_err, 0, 16);
    if (ce == cudaSuccess) ce = cudaMemcpy(b->d_taps, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(b->d_tw, tw_all.data(), sizeof(float2) * tw_all.size(), cudaMemcpyHostToDevice);
    {
        std::lock_guard<std::mutex> lk(g_beams_mu);
        g_beams.insert(b);
    }
    if (ce != cudaSuccess) {
        ppf_status s = bcuda(ce, "ppf_beams_plan: device tables");
        ppf_beams_destroy(b);
        return s;
    }
    for (int i = 0; i < n_beams; ++i) {
        b->host[i].taps = b->d_taps + taps_off[i];
        b->host[i].tw = b->d_tw + tw_off[C[i]];
    }
    ppf_status s = build_tiles(b, 1ll << 20);
    if (s != PPF_OK) {
        ppf_beams_destroy(b);
        return s;
    }
    *out = b;
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_bind(ppf_beams_t b, const void* const* in_dev, void* const* out_dev) {
    if (!valid_beams(b)) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_bind: invalid handle");
    if (in_dev == nullptr || out_dev == nullptr) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_bind: NULL table");
    for (int i = 0; i < b->n_beams; ++i) {
        if (in_dev[i] == nullptr || out_dev[i] == nullptr)
            return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_bind: beam %d: NULL buffer", i);
        if ((reinterpret_cast<uintptr_t>(in_dev[i]) | reinterpret_cast<uintptr_t>(out_dev[i])) & 15)
            return ppf::set_error(PPF_ERR_ALIGNMENT, "ppf_beams_bind: beam %d: buffers must be 16-byte aligned", i);
        b->host[i].in = in_dev[i];
        b->host[i].out = out_dev[i];
    }
    cudaError_t ce = cudaMemcpy(b->d_beams, b->host.data(), sizeof(ppf::BeamDesc) * b->n_beams, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_bind");
    b->bound = true;
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_set_tiling(ppf_beams_t b, long long tile_samples) {
    if (!valid_beams(b)) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_set_tiling: invalid handle");
    if (tile_samples < 1) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_set_tiling: tile_samples < 1");
    return build_tiles(b, tile_samples);
}

extern "C" ppf_status ppf_beams_execute(ppf_beams_t b, int ctas_per_sm, ppf_stream_t stream) {
    if (!valid_beams(b)) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_execute: invalid handle");
    if (!b->bound) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_execute: buffers not bound");
    if (ctas_per_sm < 1 || ctas_per_sm > b->occupancy) ctas_per_sm = b->occupancy;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (b->n_wide + b->n_narrow == 0) return PPF_OK;
    cudaError_t ce = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned long long), st);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_execute: queue reset");
    ppf::BeamsArgs a{b->d_beams, b->d_tiles, b->d_queue, b->d_err, b->n_wide, b->n_narrow, 0};
    long long grid = (long long)b->sms * ctas_per_sm;
    // at most one CTA per wide tile plus one per two narrow tiles is busy
    grid = std::min(grid, std::max<long long>(1, b->n_wide + (b->n_narrow + 1) / 2));
    ppf::pfb_beams_kernel<<<(int)grid, ppf::kBeamThreads, ppf::kBeamSmem, st>>>(a);
    ce = cudaPeekAtLastError();
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_execute: launch");
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_info(ppf_beams_t b, long long info[7]) {
    if (!valid_beams(b) || info == nullptr) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_info: invalid argument");
    info[0] = b->n_beams;
    info[1] = b->n_wide + b->n_narrow;
    info[2] = b->tile_samples;
    info[3] = b->occupancy;
    info[4] = b->sms;
    info[5] = ppf::kBeamSmem;
    info[6] = b->n_wide;
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_check_device(ppf_beams_t b, ppf_stream_t stream) {
    if (!valid_beams(b)) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_check_device: invalid handle");
    int v = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaMemcpyAsync(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_check_device");
    if (v != 0) {
        cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return ppf::set_error(PPF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait gave up; the launch returned early");
    }
    return PPF_OK;
}
