// ppf_bwd_unfused.cuh -- the adjoint of the PFB for every shape the forward
// plans (C = 32 .. 4096 and 3 * 2^k, T up to 64, any input type), as three
// passes over a g_y scratch in device memory.  The fused backward kernel
// (ppf_bwd.cuh) covers C in [64, 512] with T <= 16; outside that its carried
// rows and its G/x batches no longer fit one SM, so the three sums of the
// adjoint (same convention as ppf_bwd.cuh, PyTorch's conjugate Wirtinger
// gradient, G = grad_Y):
//   g_y = F^H G                                   (unnormalised inverse DFT)
//   grad_x[r][c] = sum_{t<T} h[t][c] g_y[r-t][c]  (transposed FIR, Alg. 1)
//   grad_h[t][c] = sum_s Re(conj(g_y[s][c]) x[s+t][c])
// (g_y[s] = 0 outside 0 <= s < S) run as separate kernels:
//   1. pfb_bwd_idft_kernel<C>: batches of G rows through shared memory, the
//      forward's DFT stages in their inverse mode (conj(F conj(.))), g_y rows
//      to the scratch;
//   2. pfb_bwd_gradx_kernel: one thread per channel pair and tile of kAdjL
//      raw rows, taps outermost with a window of kAdjL g_y rows in registers
//      (one new row per tap, with its tap, staged kAdjStage taps ahead);
//   3. pfb_bwd_gradh_kernel<IN>: one thread per channel pair, block of
//      kAdjTB taps and part of the rows of all streams, a window of kAdjTB
//      x rows in registers (one new x row and one g_y row per row, staged
//      kAdjStage rows ahead); per-part partial sums reduced in a fixed order
//      by pfb_bwd_reduce_kernel (deterministic).
// The staging: each thread copies the rows it will need with cp.async into
// shared-memory slots of its own and waits for the oldest group, so several
// global loads are in flight per thread without holding registers.
// HBM traffic per raw sample is about G 8 + g_y 8 (write) + g_y 8 + grad_x 8
// + g_y 8 + x; the halo and tap-block re-reads come from L2.
#pragma once

#include "ppf_fwd.cuh"

namespace ppf {

struct IdftArgs {
    const float2* gY;        // incoming gradient, n_spectra*C per stream, streams gY_stride apart
    float2* gy;              // g_y, n_spectra*C per stream, streams contiguous
    const float2* tw;        // the forward plan's twiddle tables
    long long n_spectra, gY_stride, n_streams;
};

// Threads and batch of the forward's generic kernel in its plain
// configuration (for these its DFT stages divide their items exactly):
// 64 KB of spectra per batch (48 KB for C = 384/768/1536, 96 KB at 3072).
template <int C>
struct IdftShape {
    static constexpr int NT = C >= 2048 ? 512 : 256;
    static constexpr int B = C >= 4096 ? 2 : C >= 2048 ? 4 : is_c3(C) ? 16 * 384 / C : 8192 / C;
    static constexpr int YBYTES = B * C * 8;
    static constexpr int SMEM = YBYTES + tw_size(C) * 8;
};

template <int C>
__global__ void __launch_bounds__(IdftShape<C>::NT) pfb_bwd_idft_kernel(IdftArgs a) {
    using S = IdftShape<C>;
    constexpr int NT = S::NT, B = S::B, NST = fft_stages(C);
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ybuf = reinterpret_cast<float2*>(smem);
    float2* tw_s = reinterpret_cast<float2*>(smem + S::YBYTES);
    const int tid = threadIdx.x;
    for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = a.tw[i];
    float4* y4 = reinterpret_cast<float4*>(ybuf);
    BatchShare share((a.n_spectra + B - 1) / B, a.n_streams, blockIdx.x, gridDim.x);
    long long strm, lo, hi;
    while (share.next(strm, lo, hi)) {
        const float4* src = reinterpret_cast<const float4*>(a.gY + (size_t)strm * a.gY_stride);
        float4* dst = reinterpret_cast<float4*>(a.gy + (size_t)strm * a.n_spectra * C);
        for (long long k = lo; k < hi; ++k) {
            const long long s0 = k * B;
            const int rows = (int)(a.n_spectra - s0 < B ? a.n_spectra - s0 : B);
            const long long base = s0 * (C / 2);            // float4 index of the batch's first row
            __syncthreads();   // the previous batch's rows have been stored (and the twiddles copied)
            for (int i = tid; i < B * C / 2; i += NT)
                y4[i] = (i < rows * (C / 2)) ? __ldcs(src + base + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            // inverse mode: the last stage leaves g_y rows in natural order in ybuf, then synchronises
            static_for<NST>([&](auto p) {
                fft_stage<C, B, NT, decltype(p)::value, OUT_CF32, true, 0, true>(ybuf, tw_s, nullptr, 0, 0, 0);
            });
            for (int i = tid; i < rows * (C / 2); i += NT) dst[base + i] = y4[i];
        }
    }
}

struct AdjFirArgs {
    const float2* gy;        // g_y, n_spectra*C per stream, streams contiguous
    const float* taps;       // tap-major, rows >= T zero
    float2* gx;              // grad_x, n_raw*C per stream, streams gx_stride apart
    long long n_spectra, n_streams, gx_stride;
    int C, T;
};

constexpr int kAdjL = 8;     // raw rows per grad_x tile
constexpr int kAdjStage = 8; // rows (or taps) each thread has in flight through its staging slots
constexpr int kAdjTB = 8;    // taps per grad_h block

// Complex pair (2 channels) as (re0, re1) and (im0, im1) packed registers.
__device__ __forceinline__ void load_gpair(const float2* __restrict__ row, int p, bool ok, unsigned long long& re,
                                           unsigned long long& im) {
    const float4 v = ok ? __ldg(reinterpret_cast<const float4*>(row) + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    re = pk2(v.x, v.z);
    im = pk2(v.y, v.w);
}

// grid.x: tiles (grid-stride over n_streams * ceil(n_raw / kAdjL)), grid.y: blocks of channel pairs.  Each thread
// streams the g_y rows its taps bring in, and the taps, through kAdjStage
// shared-memory staging slots of its own (cp.async), kAdjStage taps ahead.
static __global__ void __launch_bounds__(128) pfb_bwd_gradx_kernel(AdjFirArgs a) {
    constexpr int L = kAdjL, D = kAdjStage;
    static_assert(L % D == 0, "staging slots repeat within a tap block");
    __shared__ __align__(16) float4 sg[D][128];                      // g_y pair of a staged row
    __shared__ __align__(8) float2 sh[D][128];                       // taps of the pair for a staged tap
    const int C = a.C, T = a.T;
    const int tl = threadIdx.x;
    const int p = blockIdx.y * blockDim.x + tl;                      // channel pair
    if (p >= C / 2) return;
    const long long S = a.n_spectra, n_raw = S + T - 1;
    const long long tiles = (n_raw + L - 1) / L;
    const float2* taps2 = reinterpret_cast<const float2*>(a.taps);   // [t][pair]
    for (long long u = blockIdx.x; u < tiles * a.n_streams; u += gridDim.x) {
        const long long strm = u / tiles, r0 = (u - strm * tiles) * L;
        const float2* g = a.gy + (size_t)strm * S * C;
        // tap t (>= 1) brings row r0 - t (zero outside the stream) and h[t]
        // into staging slot (t - 1) mod D, requested D taps ahead
        auto stage = [&](int t) {
            if (t < T) {
                const int slot = (t - 1) % D;
                const long long r = r0 - t;
                if (r >= 0 && r < S) cp_async<16>(&sg[slot][tl], g + (size_t)r * C + 2 * p);
                else sg[slot][tl] = make_float4(0.f, 0.f, 0.f, 0.f);
                cp_async<8>(&sh[slot][tl], taps2 + (size_t)t * (C / 2) + p);
            }
            cp_async_commit();
        };
#pragma unroll
        for (int d = 1; d <= D; ++d) stage(d);
        // slot m mod L holds g_y row r0 + m; at tap t output j reads row r0 + j - t
        unsigned long long wr[L], wi[L], ar[L], ai[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const long long r = r0 + j;
            load_gpair(g + (size_t)r * C, p, r < S, wr[j], wi[j]);
            ar[j] = ai[j] = 0ull;
        }
        unsigned long long hh;
        {
            const float2 h = __ldg(taps2 + p);
            hh = pk2(h.x, h.y);
        }
        for (int tb = 0; tb < T; tb += L) {
#pragma unroll
            for (int v = 0; v < L; ++v) {
                const int t = tb + v;
                if (t < T) {
                    if (t > 0) {                                 // row r0 - t enters slot (-t) mod L
                        const int slot = (v + L - 1) % D;        // (t - 1) mod D
                        cp_async_wait<D - 1>();
                        const float4 gv = sg[slot][tl];
                        wr[(L - v) % L] = pk2(gv.x, gv.z);
                        wi[(L - v) % L] = pk2(gv.y, gv.w);
                        const float2 h = sh[slot][tl];
                        hh = pk2(h.x, h.y);
                        stage(t + D);
                    }
#pragma unroll
                    for (int j = 0; j < L; ++j) {
                        ffma2(ar[j], hh, wr[(j - v + L) % L]);
                        ffma2(ai[j], hh, wi[(j - v + L) % L]);
                    }
                }
            }
        }
        cp_async_wait<0>();
        float4* out = reinterpret_cast<float4*>(a.gx + (size_t)strm * a.gx_stride);
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const long long r = r0 + j;
            if (r < n_raw) {
                const float2 re = upk2(ar[j]), im = upk2(ai[j]);
                out[(size_t)r * (C / 2) + p] = make_float4(re.x, im.x, re.y, im.y);
            }
        }
    }
}

struct AdjCorrArgs {
    const float2* gy;        // g_y, n_spectra*C per stream, streams contiguous
    const void* x;           // forward input (plan's type), n_raw*C per stream, streams x_stride apart
    float* partials;         // n_parts rows of TM*C partial sums
    long long n_spectra, n_streams, x_stride;
    int C, T, TM, n_parts;
};


// grid.x: parts of the rows of all streams, grid.y: blocks of channel pairs,
// grid.z: blocks of kAdjTB taps.  Each thread streams its rows through kAdjStage
// shared-memory staging slots of its own (cp.async), so kAdjStage rows of g_y and x
// are in flight while it works on the oldest.
template <int IN>
__global__ void __launch_bounds__(128, 4) pfb_bwd_gradh_kernel(AdjCorrArgs a) {
    constexpr int TB = kAdjTB, BIN = InTraits<IN>::bytes, XB = 2 * BIN, D = kAdjStage;
    static_assert(TB % D == 0 || D % TB == 0, "staging slots and window slots repeat together");
    __shared__ __align__(16) float4 sg[D][128];                      // g_y pair of a staged row
    __shared__ __align__(16) unsigned char sx[D][128 * XB];          // x pair of a staged row
    const int C = a.C, T = a.T;
    const int tl = threadIdx.x;
    const int p = blockIdx.y * blockDim.x + tl;                      // channel pair
    const bool active = p < C / 2;
    const int t0 = blockIdx.z * TB;
    const long long S = a.n_spectra, n_raw = S + T - 1;
    const long long R = S * a.n_streams;
    long long u = (long long)blockIdx.x * R / a.n_parts;
    const long long u1 = (long long)(blockIdx.x + 1) * R / a.n_parts;
    unsigned long long acc[TB];
#pragma unroll
    for (int v = 0; v < TB; ++v) acc[v] = 0ull;
    auto unpack_x = [&](const unsigned char* q, unsigned long long& re, unsigned long long& im) {
        const float4 v = load_pair_smem<IN>(q);
        re = pk2(v.x, v.z);
        im = pk2(v.y, v.w);
    };
    while (active && u < u1) {                                        // segments of single streams
        const long long strm = u / S, s0 = u - strm * S;
        const long long s1 = (u1 - strm * S < S) ? u1 - strm * S : S;
        u = strm * S + s1;
        const float2* g = a.gy + (size_t)strm * S * C;
        const unsigned char* x = static_cast<const unsigned char*>(a.x) + (size_t)strm * a.x_stride * BIN;
        // stage row s: g_y row s and the x row entering the window there, s + t0 + TB - 1
        auto stage = [&](long long s, int slot) {
            if (s < s1) {
                cp_async<16>(&sg[slot][tl], g + (size_t)s * C + 2 * p);
                const long long r = s + t0 + TB - 1;
                if (r < n_raw) {
                    cp_async<XB>(&sx[slot][tl * XB], x + ((size_t)r * C + 2 * p) * BIN);
                } else {
                    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    memcpy(&sx[slot][tl * XB], &z, XB);
                }
            }
            cp_async_commit();
        };
        // slot m mod TB holds x row s0 + t0 + m (re pair, im pair); at row s0 + i,
        // tap t0 + v reads row s0 + i + t0 + v, slot (i + v) mod TB
        unsigned long long xr[TB], xi[TB];
#pragma unroll
        for (int m = 0; m + 1 < TB; ++m) {
            const long long r = s0 + t0 + m;
            const float4 v = r < n_raw ? load_pair_global<IN>(x, r * C + 2 * p) : make_float4(0.f, 0.f, 0.f, 0.f);
            xr[m] = pk2(v.x, v.z);
            xi[m] = pk2(v.y, v.w);
        }
#pragma unroll
        for (int d = 0; d < D; ++d) stage(s0 + d, d);
        for (long long ib = 0; ib < s1 - s0; ib += TB) {
#pragma unroll
            for (int i = 0; i < TB; ++i) {
                const long long s = s0 + ib + i;
                if (s < s1) {
                    const int slot = i % D;                           // (s - s0) mod D
                    cp_async_wait<D - 1>();                           // row s has landed
                    const float4 gv = sg[slot][tl];
                    const unsigned long long gr = pk2(gv.x, gv.z), gi = pk2(gv.y, gv.w);
                    unpack_x(&sx[slot][tl * XB], xr[(i + TB - 1) % TB], xi[(i + TB - 1) % TB]);
                    stage(s + D, slot);
#pragma unroll
                    for (int v = 0; v < TB; ++v) {
                        ffma2(acc[v], gr, xr[(i + v) % TB]);
                        ffma2(acc[v], gi, xi[(i + v) % TB]);
                    }
                }
            }
        }
        cp_async_wait<0>();
    }
    if (!active) return;
    float* part = a.partials + (size_t)blockIdx.x * a.TM * C;
#pragma unroll
    for (int v = 0; v < TB; ++v) {
        const int t = t0 + v;
        if (t < T) {
            const float2 s = upk2(acc[v]);
            *reinterpret_cast<float2*>(part + (size_t)t * C + 2 * p) = s;
        }
    }
}

struct IdftInfo {
    int threads, batch, smem;
    const void* fn;
};

template <int C>
inline IdftInfo idft_info() {
    return IdftInfo{IdftShape<C>::NT, IdftShape<C>::B, IdftShape<C>::SMEM,
                    reinterpret_cast<const void*>(&pfb_bwd_idft_kernel<C>)};
}

template <int C>
inline cudaError_t idft_launch(const IdftArgs& a, int grid, cudaStream_t st) {
    pfb_bwd_idft_kernel<C><<<grid, IdftShape<C>::NT, IdftShape<C>::SMEM, st>>>(a);
    return cudaPeekAtLastError();
}

}  // namespace ppf
