// ppf_fwd.cuh -- the fused polyphase filter bank forward kernel.
//
// One persistent CTA loops over batches of B consecutive output spectra.
// Per batch:
//   1. FIR (Alg. 1): each thread owns a channel pair and a segment of L
//      output spectra; it streams the L+T-1 raw samples of its pair from
//      global memory (each raw sample is converted to FP32 once per segment
//      and reused by all T taps in registers; the T-1 spectra shared with
//      the neighbouring segment -- the halo of Sec. 3.2 -- come from L2),
//      and writes the filtered spectra y to shared memory.  y never goes to
//      global memory.
//   2. DFT (Eq. 2) of every filtered spectrum, C = R_0 * R_1 * ... as a
//      sequence of stages.  Stage p does R_p-point DFTs in registers on
//      columns of stride N_{p+1} = N_p / R_p, multiplies by the twiddles
//      W_{N_p}^{b k}, and writes the result back to shared memory in the
//      layout the next stage reads; the last stage writes the frequency
//      spectrum to global memory in natural bin order with coalesced
//      streaming stores.
//
// Index bookkeeping of the stages (all per spectrum):
//   A_p(prefix, j), j in [0, N_p): prefix = (k_0, ..., k_{p-1}) linearised
//   with k_0 fastest.  Stage p item (prefix, b), b in [0, N_{p+1}):
//     reads  A_p(prefix, N_{p+1} a + b),           a   in [0, R_p)
//     writes A_{p+1}(prefix + P_p k, b),           k   in [0, R_p), P_p = C / N_p
//   and finally A_P(q) = Y[q] (q = k_0 + R_0 k_1 + ...).
#pragma once

#include "ppf_device.cuh"

namespace ppf {

// -------------------------------------------------------------- FFT plan
constexpr int fft_stages(int C) { return C >= 2048 ? 3 : 2; }
constexpr int fft_radix(int C, int p) {
    switch (C) {
        case 32:   return p == 0 ? 8 : 4;
        case 64:   return 8;
        case 128:  return p == 0 ? 16 : 8;
        case 256:  return 16;
        case 512:  return p == 0 ? 32 : 16;
        case 1024: return 32;
        case 2048: return p < 2 ? 16 : 8;
        case 4096: return 16;
        default:   return 0;
    }
}
// N_p = R_p * R_{p+1} * ... (N_0 = C, N_P = 1)
constexpr int fft_n(int C, int p) {
    int n = 1;
    for (int q = p; q < fft_stages(C); ++q) n *= fft_radix(C, q);
    return n;
}
// Padded physical index inside one spectrum slot for buffer A_p.
// A_0 (the FIR output) is unpadded; later buffers get one pad element every
// G elements so strided column reads do not collide in shared-memory banks.
constexpr int pad_group(int C, int p) {
    return p == fft_stages(C) - 1 ? (fft_radix(C, p) > 16 ? fft_radix(C, p) : 16) : 16;
}
template <int C, int P>
__device__ __forceinline__ int phys(int i) {
    if constexpr (P == 0) return i;
    else return i + i / pad_group(C, P);
}
// Floats2 per spectrum slot (even, so float4 stores of y stay aligned).
constexpr int slot_size(int C) { return C + C / 16; }
// Twiddle table offsets: stage p (p < P-1) holds W_{N_p}^{b k} at [k*N_{p+1} + b].
constexpr int tw_offset(int C, int p) {
    int off = 0;
    for (int q = 0; q < p; ++q) off += fft_n(C, q);
    return off;
}
constexpr int tw_size(int C) { return tw_offset(C, fft_stages(C) - 1); }

// ------------------------------------------------------------ launch shape
template <int C, int TM, int IN>
struct FwdShape {
    static constexpr int NT = C >= 2048 ? 512 : 256;                 // threads per CTA
    static constexpr int PAIRS = C / 2;
    static constexpr int B = (C >= 4096) ? 2 : (C >= 2048) ? 4 : 8192 / C;   // spectra per batch
    static constexpr int L0 = TM >= 32 ? 8 : 16;
    static constexpr int L = L0 < B ? L0 : B;                        // FIR segment (outputs)
    static constexpr int G = B / L;                                  // segments per batch
    static constexpr int FIR_ITEMS = PAIRS * G;                      // (pair, segment) items
    static constexpr int FPT = FIR_ITEMS / NT;                       // FIR items per thread
    static constexpr int SLOT = slot_size(C);
    static constexpr int SMEM = (B * SLOT + tw_size(C)) * 8;         // dynamic smem bytes
    // each thread keeps one channel pair for the whole run: taps stay in registers
    static constexpr bool TAPS_IN_REGS = (FPT == 1) && (TM <= 16) && (NT % PAIRS == 0);
    static_assert(FPT * NT == FIR_ITEMS && FPT >= 1, "FIR items must divide evenly");
};

struct FwdArgs {
    const void* in;          // raw stream, C*(n_spectra+T-1) samples
    void* out;               // n_spectra*C outputs
    const float* taps;       // TM*C floats, tap-major, rows >= T are zero
    const float2* tw;        // twiddle tables, tw_size(C) entries
    long long n_spectra;
    int T;
};

// One FFT stage over the whole batch held in shared memory.
template <int C, int B, int NT, int P, int OUT>
__device__ __forceinline__ void fft_stage(float2* __restrict__ ybuf, const float2* __restrict__ tws,
                                          void* __restrict__ out, long long sb, long long n_spectra) {
    constexpr int NST = fft_stages(C);
    constexpr int R = fft_radix(C, P);
    constexpr int NP = fft_n(C, P);
    constexpr int NN = NP / R;                 // N_{p+1}
    constexpr int PP = C / NP;                 // prefixes at this stage
    constexpr int ITEMS = C / R;               // items per spectrum
    constexpr int IPT = B * ITEMS / NT;        // items per thread
    constexpr int SLOT = slot_size(C);
    static_assert(IPT * NT == B * ITEMS, "items must divide evenly");
    const int tid = threadIdx.x;

    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = tid + it * NT;
        const int sp = item / ITEMS, e = item % ITEMS;
        const int b = e % NN, prefix = e / NN;
        const float2* src = ybuf + sp * SLOT;
#pragma unroll
        for (int a = 0; a < R; ++a) v[it][a] = src[phys<C, P>(prefix * NP + NN * a + b)];
    }
    __syncthreads();   // every read of this stage is done before anything is overwritten
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = tid + it * NT;
        const int sp = item / ITEMS, e = item % ITEMS;
        const int b = e % NN, prefix = e / NN;
        dft_reg<R>(v[it]);
        if constexpr (P + 1 < NST) {
            const float2* twp = tws + tw_offset(C, P);
#pragma unroll
            for (int k = 1; k < R; ++k) v[it][k] = cmul(v[it][k], twp[k * NN + b]);
            float2* dst = ybuf + sp * SLOT;
#pragma unroll
            for (int k = 0; k < R; ++k) dst[phys<C, P + 1>((prefix + PP * k) * NN + b)] = v[it][k];
        } else {
            const long long s = sb + sp;
            if (s < n_spectra) {
#pragma unroll
                for (int k = 0; k < R; ++k) store_out<OUT>(out, s * C + prefix + PP * k, v[it][k]);
            }
        }
    }
    if constexpr (P + 1 < NST) __syncthreads();
}

__device__ __forceinline__ void fma_pair(float4& acc, float2 h, float4 x) {
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.y = fmaf(h.x, x.y, acc.y);
    acc.z = fmaf(h.y, x.z, acc.z);
    acc.w = fmaf(h.y, x.w, acc.w);
}

template <int C, int IN>
__device__ __forceinline__ float4 load_raw(const void* in, long long r, long long n_raw, int cp) {
    return (r < n_raw) ? load_pair_global<IN>(in, r * C + 2 * cp) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// FIR (Alg. 1) of channel pair cp for the L output spectra r0 .. r0+L-1:
//   acc[j] = sum_{t<T} h[t][cp] * x[r0 + j + t][cp]
// Every raw sample of the segment (L+T-1 of them) is loaded and converted
// once; the taps are applied in ascending t for every output.
template <int C, int TM, int IN, int L, int PAIRS, bool TAPS_IN_REGS>
__device__ __forceinline__ void fir_segment(const void* __restrict__ in, const float2* __restrict__ taps2,
                                            const float2 (&hreg)[TAPS_IN_REGS ? TM : 1], int cp,
                                            long long r0, long long n_raw, int T, float4 (&acc)[L]) {
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (TM <= 16) {
        // raw-sample-outer order: all TM taps live in registers, one sample live.
        float2 h[TM];
#pragma unroll
        for (int t = 0; t < TM; ++t) {
            if constexpr (TAPS_IN_REGS) h[t] = hreg[t];
            else h[t] = __ldg(taps2 + t * PAIRS + cp);
        }
#pragma unroll
        for (int i = 0; i < L + TM - 1; ++i) {
            if (i < L + T - 1) {
                const float4 x = load_raw<C, IN>(in, r0 + i, n_raw, cp);
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int t = i - j;
                    if (t >= 0 && t < TM) {
                        if constexpr (IN == IN_CF32) {
                            if (t < T) fma_pair(acc[j], h[t], x);   // keeps inf/NaN out of unrelated outputs
                        } else {
                            fma_pair(acc[j], h[t], x);             // taps t >= T are zero
                        }
                    }
                }
            }
        }
    } else {
        // Large T: tap-outer order with a circular window of L samples
        // (slot (i mod L) holds raw sample r0+i), T is a runtime loop bound.
        // After tap t the sample r0+t is dead and its slot is refilled with
        // r0+t+L, L taps before it is needed.  Live: L accumulators + L samples.
        float4 xw[L];
#pragma unroll
        for (int i = 0; i < L; ++i) xw[i] = load_raw<C, IN>(in, r0 + i, n_raw, cp);
#pragma unroll 1
        for (int tb = 0; tb < T; tb += L) {
#pragma unroll
            for (int u = 0; u < L; ++u) {
                const int t = tb + u;
                if (t < T) {
                    const float2 h = __ldg(taps2 + t * PAIRS + cp);
#pragma unroll
                    for (int j = 0; j < L; ++j) fma_pair(acc[j], h, xw[(j + u) % L]);
                    if (t + 1 < T) xw[u] = load_raw<C, IN>(in, r0 + t + L, n_raw, cp);
                }
            }
        }
    }
}

template <int C, int TM, int IN, int OUT>
__global__ void __launch_bounds__(FwdShape<C, TM, IN>::NT, FwdShape<C, TM, IN>::NT == 256 ? 2 : 1)
pfb_fwd_kernel(FwdArgs args) {
    using S = FwdShape<C, TM, IN>;
    constexpr int NT = S::NT, B = S::B, L = S::L, SLOT = S::SLOT;
    constexpr int NST = fft_stages(C);
    extern __shared__ float4 smem_f4[];
    float2* ybuf = reinterpret_cast<float2*>(smem_f4);
    float2* tws = ybuf + B * SLOT;

    const int tid = threadIdx.x;
    const long long n_spectra = args.n_spectra;
    const long long n_raw = n_spectra + args.T - 1;
    const int T = args.T;
    const long long nbatch = (n_spectra + B - 1) / B;

    for (int i = tid; i < tw_size(C); i += NT) tws[i] = args.tw[i];

    // FIR work assignment: item = tid + k*NT -> pair cp = item % PAIRS, segment g = item / PAIRS.
    const float2* taps2 = reinterpret_cast<const float2*>(args.taps);   // [t][pair]
    float2 hreg[S::TAPS_IN_REGS ? TM : 1];
    if constexpr (S::TAPS_IN_REGS) {
#pragma unroll
        for (int t = 0; t < TM; ++t) hreg[t] = __ldg(taps2 + t * S::PAIRS + tid % S::PAIRS);
    }
    __syncthreads();

    for (long long batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
        const long long sb = batch * B;             // first output spectrum of the batch
        // ---------------------------------------------------------- FIR
#pragma unroll 1
        for (int k = 0; k < S::FPT; ++k) {
            const int item = tid + k * NT;
            const int cp = item % S::PAIRS, g = item / S::PAIRS;
            const long long r0 = sb + g * L;        // first raw spectrum of the segment
            float4 acc[L];
            fir_segment<C, TM, IN, L, S::PAIRS, S::TAPS_IN_REGS>(args.in, taps2, hreg, cp, r0, n_raw, T, acc);
#pragma unroll
            for (int j = 0; j < L; ++j)
                *reinterpret_cast<float4*>(ybuf + (g * L + j) * SLOT + 2 * cp) = acc[j];
        }
        __syncthreads();
        // ---------------------------------------------------------- FFT
        static_for<NST>([&](auto p) {
            fft_stage<C, B, NT, decltype(p)::value, OUT>(ybuf, tws, args.out, sb, n_spectra);
        });
    }
}

// Host side: shape + launch of one instantiation.
struct FwdInfo {
    int threads, batch, smem, stages, tap_bucket;
    const void* fn;
};

template <int C, int TM, int IN, int OUT>
inline FwdInfo fwd_info() {
    using S = FwdShape<C, TM, IN>;
    return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM,
                   reinterpret_cast<const void*>(&pfb_fwd_kernel<C, TM, IN, OUT>)};
}

template <int C, int TM, int IN, int OUT>
inline cudaError_t fwd_launch(const FwdArgs& a, int grid, cudaStream_t st) {
    using S = FwdShape<C, TM, IN>;
    pfb_fwd_kernel<C, TM, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    return cudaPeekAtLastError();
}

// Twiddle table contents (host, FP64 -> FP32): stage p < P-1 holds
// W_{N_p}^{b k} = exp(-2 pi i b k / N_p) at [tw_offset(p) + k*N_{p+1} + b].
template <int C>
inline void fill_twiddles(float2* host) {
    for (int p = 0; p + 1 < fft_stages(C); ++p) {
        const int NP = fft_n(C, p), R = fft_radix(C, p), NN = NP / R;
        for (int k = 0; k < R; ++k)
            for (int b = 0; b < NN; ++b) {
                const long e = (long)b * k % NP;
                host[tw_offset(C, p) + k * NN + b] =
                    make_float2((float)cos2pi(e, NP), (float)(-sin2pi(e, NP)));
            }
    }
}

}  // namespace ppf
