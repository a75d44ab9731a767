// ppf_beams.cu -- many independent beams with uneven channel counts, taps and
// spectrum counts in ONE persistent launch.
//
// The plan cuts every beam into tiles (contiguous ranges of output batches of
// about `tile_samples` samples) and sorts all tiles largest first.  The grid
// is persistent (CTAs per SM x SMs); each CTA pulls the next tile index from
// a device counter (reset by a memset node before every launch, so the pair
// can be captured in a CUDA graph), reads the tile's beam descriptor and runs
// the FIR + DFT of that range with the code of the beam's (C, tap bucket)
// class.  All classes share one block size (256 threads) and one dynamic
// shared-memory size (the largest class's).  Beams with C >= 2048 instead
// run, after the persistent launch and on the same stream, one launch each of
// the single-stream kernel ppf_execute uses for their shape (a thread-block
// cluster kernel or the generic one, with the grid the GPU holds at once).
// Complex int8 input, complex FP32 output: the multi-beam workload of the
// channeliser.
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

namespace ppf {

constexpr int kBeamThreads = 256;
constexpr int kBeamC[] = {64, 128, 256, 512, 1024, 2048, 4096};
constexpr int kBeamTM[] = {4, 8, 16};
constexpr int kNumC = 7, kNumTM = 3;

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
    const BeamTile* tiles;
    unsigned long long* queue;   // next tile index
    int* err;
    long long n_tiles;
    int flags;
};

template <int CI, int TI>
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
    return fwd_range<C, TM, IN_CI8, OUT_CF32, kBeamThreads>(fa, d.in, d.out, t.lo, t.hi, smem);
}

template <int CI, int TI>
__device__ __forceinline__ bool beam_dispatch(int cls, const BeamsArgs& a, const BeamDesc& d, const BeamTile& t,
                                              unsigned char* smem) {
    if (cls == CI * kNumTM + TI) return beam_tile<CI, TI>(a, d, t, smem);
    if constexpr (TI + 1 < kNumTM) return beam_dispatch<CI, TI + 1>(cls, a, d, t, smem);
    else if constexpr (CI + 1 < kNumC) return beam_dispatch<CI + 1, 0>(cls, a, d, t, smem);
    else return true;
}

__global__ void __launch_bounds__(kBeamThreads, 2) pfb_beams_kernel(BeamsArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1ull);
        __syncthreads();
        const unsigned long long ti = s_tile;
        __syncthreads();
        if (ti >= (unsigned long long)a.n_tiles) return;
        const BeamTile t = a.tiles[ti];
        const BeamDesc d = a.beams[t.beam];
        if (!beam_dispatch<0, 0>(d.cls, a, d, t, smem)) return;
    }
}

template <int CI, int TI>
constexpr int class_smem() {
    constexpr int s = FwdShape<kBeamC[CI], kBeamTM[TI], IN_CI8, kBeamThreads>::SMEM;
    if constexpr (TI + 1 < kNumTM) return s > class_smem<CI, TI + 1>() ? s : class_smem<CI, TI + 1>();
    else if constexpr (CI + 1 < kNumC) return s > class_smem<CI + 1, 0>() ? s : class_smem<CI + 1, 0>();
    else return s;
}
template <int CI, int TI>
constexpr int class_batch(int cls) {
    if (cls == CI * kNumTM + TI) return FwdShape<kBeamC[CI], kBeamTM[TI], IN_CI8, kBeamThreads>::B;
    if constexpr (TI + 1 < kNumTM) return class_batch<CI, TI + 1>(cls);
    else if constexpr (CI + 1 < kNumC) return class_batch<CI + 1, 0>(cls);
    else return 0;
}
constexpr int kBeamSmem = class_smem<0, 0>();

// twiddles of every supported C (host)
void fill_beam_twiddles(int C, std::vector<float2>& tw) {
    switch (C) {
#define PPF_BTW(CC) case CC: tw.assign(tw_size(CC) > 0 ? tw_size(CC) : 1, make_float2(0.f, 0.f)); fill_twiddles<CC>(tw.data()); break;
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

// The single-stream kernel of a beam that runs on its own launch (C >= 2048).
bool separate_entry(int C, int T, ppf::FwdEntry* e) {
    const int tm = T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : T <= 8 ? 8 : 16;
    if (C == 2048) return ppf::fwd_lookup_c2048(tm, PPF_IN_CI8, PPF_OUT_CF32, e);
    if (C == 4096) return ppf::fwd_lookup_c4096(tm, PPF_IN_CI8, PPF_OUT_CF32, e);
    return false;
}

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
    std::vector<int> big;                  // beams run by a launch of their own
    std::vector<ppf::FwdEntry> big_entry;  // their kernels
    std::vector<int> big_units;            // resident work units (CTAs or clusters) of each
    ppf::BeamDesc* d_beams;
    ppf::BeamTile* d_tiles;
    long long n_tiles;
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

static ppf_status build_tiles(ppf_beams_t b, long long tile_samples) {
    std::vector<ppf::BeamTile> tiles;
    std::vector<long long> weight;
    std::vector<bool> is_big(b->n_beams, false);
    for (int i : b->big) is_big[i] = true;
    for (int i = 0; i < b->n_beams; ++i) {
        if (is_big[i]) continue;
        const ppf::BeamDesc& d = b->host[i];
        const long long B = ppf::class_batch<0, 0>(d.cls);
        const long long nbt = (d.n_spectra + B - 1) / B;
        long long per = tile_samples / (B * d.C);
        if (per < 1) per = 1;
        for (long long lo = 0; lo < nbt; lo += per) {
            const long long hi = std::min(nbt, lo + per);
            tiles.push_back(ppf::BeamTile{lo, hi, i});
            weight.push_back((hi - lo) * B * d.C * (long long)b->tm[i]);
        }
    }
    std::vector<size_t> order(tiles.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return weight[x] > weight[y]; });
    std::vector<ppf::BeamTile> sorted(tiles.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = tiles[order[i]];
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    cudaError_t ce = cudaMalloc(&b->d_tiles, sizeof(ppf::BeamTile) * std::max<size_t>(1, sorted.size()));
    if (ce == cudaSuccess)
        ce = cudaMemcpy(b->d_tiles, sorted.data(), sizeof(ppf::BeamTile) * sorted.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bcuda(ce, "ppf_beams: tiles");
    b->n_tiles = (long long)sorted.size();
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
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_queue, sizeof(unsigned long long));
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
        ppf::FwdEntry e{};
        if (!separate_entry(C[i], T[i], &e)) continue;
        int units = 0;
        ce = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem);
        if (ce == cudaSuccess) {
            if (e.cluster > 0) {
                ce = ppf::max_active_clusters(e, sms, &units);
            } else {
                ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&units, e.fn, e.threads, e.smem);
                units *= sms;
            }
        }
        if (ce != cudaSuccess) {
            ppf_status s = bcuda(ce, "ppf_beams_plan: single-beam kernel");
            ppf_beams_destroy(b);
            return s;
        }
        if (units < 1) continue;      // stays on the persistent kernel
        b->big.push_back(i);
        b->big_entry.push_back(e);
        b->big_units.push_back(units);
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
    cudaError_t ce = cudaSuccess;
    if (b->n_tiles > 0) {
        ce = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), st);
        if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_execute: queue reset");
        ppf::BeamsArgs a{b->d_beams, b->d_tiles, b->d_queue, b->d_err, b->n_tiles, 0};
        long long grid = (long long)b->sms * ctas_per_sm;
        if (grid > b->n_tiles) grid = b->n_tiles;
        ppf::pfb_beams_kernel<<<(int)grid, ppf::kBeamThreads, ppf::kBeamSmem, st>>>(a);
        ce = cudaPeekAtLastError();
        if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_execute: launch");
    }
    for (size_t j = 0; j < b->big.size(); ++j) {
        const ppf::BeamDesc& d = b->host[b->big[j]];
        const ppf::FwdEntry& e = b->big_entry[j];
        ppf::FwdArgs fa;
        fa.in = d.in;
        fa.out = d.out;
        fa.in_stride = 0;
        fa.out_stride = 0;
        const long long nb = (d.n_spectra + e.batch - 1) / e.batch;
        fa.n_streams = 1;
        const long long units = std::min<long long>(b->big_units[j], nb);
        const int per_unit = e.cluster > 0 ? e.cluster : 1;
        fa.taps = d.taps;
        fa.tw = d.tw;
        fa.err = b->d_err;
        fa.n_spectra = d.n_spectra;
        fa.T = d.T;
        fa.flags = 0;
        ce = e.launch(fa, (int)(units * per_unit), st);
        if (ce != cudaSuccess) return bcuda(ce, "ppf_beams_execute: single-beam launch");
    }
    return PPF_OK;
}

extern "C" ppf_status ppf_beams_info(ppf_beams_t b, long long info[7]) {
    if (!valid_beams(b) || info == nullptr) return ppf::set_error(PPF_ERR_INVALID_ARG, "ppf_beams_info: invalid argument");
    info[0] = b->n_beams;
    info[1] = b->n_tiles;
    info[2] = b->tile_samples;
    info[3] = b->occupancy;
    info[4] = b->sms;
    info[5] = ppf::kBeamSmem;
    info[6] = (long long)b->big.size();
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
