// ppf_fwd_carry.cuh -- fused PFB forward kernel with the FIR halo carried in
// registers (used where each thread keeps one channel pair for the whole run).
//
// The raw stream of a CTA's contiguous range passes through a double-buffered
// TMA ring: slot k%2 holds raw spectra [(lo+k)B, (lo+k)B + B).  The T-1 raw
// spectra an output batch needs from before its slot (the overlap of
// neighbouring blocks, Sec. 3.2) are the last T-1 rows the same thread
// converted in the previous batch, kept in registers.  So every raw sample
// is read from HBM once, copied to shared memory once, loaded and converted
// by one thread once, and the copy of batch k+1 has a whole batch of compute
// (FIR k and the FFT of k) to land.  Because of the carry, batch k produces
// output spectra (lo+k)B - (T-1) .. (lo+k)B + B - T; the CTA processes
// nb + 1 raw batches and stores only the outputs of its own range.  (Slots
// shifted by T-1 rows, so that no halo-only batch is needed, measured 1.4 %
// slower at C = 512, T = 8, int8; a loop unrolled by two batches that
// alternates two register sets for the carried rows instead of copying them
// spilled registers.)
//
// The FIR uses packed FP32 pairs (fma.rn.f32x2): (re, im) of a sample times
// its (h, h) tap in one instruction.
#pragma once

#include <type_traits>

#include "ppf_fwd.cuh"

// The last DFT stage's buffer uses the pair-chunk swizzle (phys, LAYOUT 2)
// where it measured faster than the element swizzle: C = 1024 (+0.4 % at
// T = 8, +3 % at T = 16, int8), int16 input at C = 512 (+1.3 %) and int8
// input at C = 256 (+1.6 %); it measured 1-3 % slower for int8 and fp32 input
// at C = 512 and fp32 at C = 256.  PPF_LAYOUT2=0 turns it off.
#ifndef PPF_LAYOUT2
#define PPF_LAYOUT2 1
#endif

namespace ppf {

// every FFT stage must give each thread a whole number (>= 1) of items
constexpr bool fft_items_fit(int C, int B, int NT) {
    for (int p = 0; p < fft_stages(C); ++p) {
        const int items = B * (C / fft_radix(C, p));
        if (items < NT || items % NT != 0) return false;
    }
    return true;
}
// warp-local stages with SPW spectra per warp: every stage either fills the
// warp with whole items per lane or leaves lanes idle (fewer than 32 items),
// and no lane holds more than 64 floats of data
constexpr bool warp_fft_ok(int C, int SPW) {
    for (int p = 0; p < fft_stages(C); ++p) {
        const int R = fft_radix(C, p);
        const int items = SPW * (C / R);
        if (items >= 32 && items % 32 != 0) return false;
        const int ipt = (items + 31) / 32;
        if (ipt * R * 2 > 64) return false;
    }
    return true;
}

// Launch shape of the carry kernel for a batch of B spectra.
template <int C, int TM, int IN, int B_>
struct CarryCand {
    static constexpr int NT = C / 2;                                 // one channel pair per thread
    static constexpr int B = B_;
    static constexpr int BIN = InTraits<IN>::bytes;
    // last DFT stage's buffer: padded rows (no per-access index arithmetic)
    // where they measured faster -- C <= 128, and 16 taps at C <= 256 --
    // else the element XOR swizzle (C = 512/1024 at T <= 8 lost 2-4 % with
    // padding) or, where it measured faster, the pair-chunk swizzle
    static constexpr bool PAIR_SWIZZLE = PPF_LAYOUT2 && last_radix(C) >= 16 &&
                                         (C == 1024 || (C == 512 && IN == IN_CI16) || (C == 256 && IN == IN_CI8));
    static constexpr int LAYOUT = (C <= 128 || (TM >= 16 && C <= 256)) ? 1 : PAIR_SWIZZLE ? 2 : 0;
    static constexpr int YSPAN = spec_span<C, LAYOUT>();             // elements per spectrum in ybuf
    static constexpr int YBYTES = B * YSPAN * 8;
    static constexpr int SLOTB = B * C * BIN;
    static constexpr int TWBYTES = tw_size(C) * 8;
    static constexpr int BASE = YBYTES + 2 * SLOTB + 64;
    // registers of the FIR state (accumulators, carried rows, (h, h) taps)
    static constexpr int REGS_EST = 4 * B + 4 * (TM - 1) + 4 * TM + 4;
    static constexpr int REGS = REGS_EST <= 64 ? 64 : REGS_EST <= 80 ? 80 : REGS_EST <= 96 ? 96
                              : REGS_EST <= 128 ? 128 : REGS_EST <= 168 ? 168 : 255;
    static constexpr int SMEM_PER_SM = 228 * 1024;
    static constexpr int CTAS_REG = 65536 / (NT * REGS);
    static constexpr int CTAS_SMEM = SMEM_PER_SM / (BASE + TWBYTES + 1024);
    static constexpr int CTAS_THR = 2048 / NT < 32 ? 2048 / NT : 32;
    static constexpr int M1 = CTAS_REG < CTAS_SMEM ? CTAS_REG : CTAS_SMEM;
    static constexpr int M2 = M1 < CTAS_THR ? M1 : CTAS_THR;
    static constexpr int MINB = M2 < 1 ? 1 : M2;                     // CTAs per SM
    static constexpr int CTA_SMEM_CAP = SMEM_PER_SM / MINB - 1024 - 128;
    static constexpr int CTA_SMEM_MAX = CTA_SMEM_CAP < 226 * 1024 ? CTA_SMEM_CAP : 226 * 1024;
    static constexpr bool TW_SMEM = BASE + TWBYTES <= CTA_SMEM_MAX;
    static constexpr int RING_OFF = YBYTES + (TW_SMEM ? TWBYTES : 0);
    static constexpr int SMEM = RING_OFF + 2 * SLOTB + 64;
    static constexpr int NWARP = NT >= 32 ? NT / 32 : 1;
    static constexpr int SPW = B / NWARP;                            // spectra per warp in the FFT
    static constexpr bool OK = (C >= 64 && C <= 1024) && (NT % 32 == 0) && (TM <= 16) && (B >= TM - 1) &&
                               SMEM <= CTA_SMEM_MAX && SPW >= 1 && SPW * NWARP == B && warp_fft_ok(C, SPW);
    static constexpr int SCORE = OK ? MINB * NT : 0;                 // resident threads per SM
};

template <class A, class X>
struct better_cand {
    using type = typename std::conditional<(X::SCORE > A::SCORE), X, A>::type;
};

// The carry kernel's shape.  Batches of 16 spectra wherever they fit: the
// more resident threads per SM that smaller batches allow did not pay for
// their per-batch overhead (C = 64 int8 T = 8: 561 GS/s with 16 spectra vs
// 379 with 8; C = 256 int16 T = 4: 494 vs 172; C = 128 fp32 T = 4: 377 vs
// 267; at C = 512 smaller batches spill).  Two exceptions keep the batch
// with the most resident threads per SM (the larger on ties): int8 at
// C = 128 with 5-8 taps (483 vs 468 GS/s), and fp32 at C = 256 where 16
// spectra leave one CTA per SM.
template <int C, int TM, int IN>
struct CarryShapeSel {
    using C16 = CarryCand<C, TM, IN, 16>;
    using Best = typename better_cand<typename better_cand<C16, CarryCand<C, TM, IN, 8>>::type,
                                      CarryCand<C, TM, IN, 4>>::type;
    static constexpr bool KEEP16 = C16::OK && !(C == 128 && IN == IN_CI8 && TM == 8) &&
                                   !(C == 256 && IN == IN_CF32 && C16::MINB < 2);
    using type = typename std::conditional<KEEP16, C16, Best>::type;
};
template <int C, int TM, int IN>
struct CarryShape : CarryShapeSel<C, TM, IN>::type {};

// The carry kernel's body over output batches [lo, hi) of one stream (in,
// out: that stream's buffers), run by the thread group GRP of S::NT threads
// on its shared memory.  MULTI: the group runs several ranges in one launch
// (the multi-beam kernel): it waits for the group before reusing shared
// memory, and retires the ring's barriers after the range (every copy has
// landed by then: each issued batch is waited for) so the next range can
// initialise them again.  Returns false if a bounded wait gave up.
//
// FIRONLY: the unfused ablation -- the FIR alone, writing the filtered
// spectra y (complex FP32, spectrum-major) to global memory instead of
// transforming them (the paper's FIR kernel followed by a separate DFT).
template <int C, int TM, int IN, int OUT, bool FIRONLY, class GRP, bool MULTI>
__device__ __forceinline__ bool carry_range(const FwdArgs& args, const void* in, void* out, long long lo, long long hi,
                                            unsigned char* smem) {
    using S = CarryShape<C, TM, IN>;
    constexpr int NT = S::NT, B = S::B, BIN = S::BIN;
    constexpr int NST = fft_stages(C);
    static_assert(S::OK, "shape not supported by the carry kernel");
    float2* ybuf = reinterpret_cast<float2*>(smem);
    float2* tw_s = reinterpret_cast<float2*>(smem + S::YBYTES);
    unsigned char* ring = smem + S::RING_OFF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + 2 * S::SLOTB);     // 3 barriers
    volatile int* sflag = reinterpret_cast<volatile int*>(bars + 3);

    const int tid = GRP::tid();
    const int cp = tid;                              // channel pair
    const long long n_spectra = args.n_spectra;
    const int T = args.T;
    const int D = TM - T;                            // leading zero taps of the bucket
    const long long n_raw = n_spectra + T - 1;
    const long long nb = hi - lo;
    if (nb <= 0) return true;
    if constexpr (MULTI) GRP::sync();                // the group's previous range is done with shared memory
    const long long vlo = lo * B, vhi = (hi * B < n_spectra) ? hi * B : n_spectra;
    const long long nraw_b = (T > 1) ? nb + 1 : nb;  // raw batches this range streams
    auto rows_of = [&](long long j) -> long long {
        const long long r = n_raw - (lo + j) * B;
        return r <= 0 ? 0 : (r < B ? r : B);
    };
    auto issue = [&](long long j) {
        const long long rows = rows_of(j);
        if (rows > 0) {
            uint64_t* bar = &bars[j & 1];
            const uint32_t bytes = (uint32_t)(rows * C * BIN);
            mbar_expect_tx(bar, bytes);
            if constexpr (PPF_TMA_EVICT_FIRST)
                tma_load_1d_once(ring + (j & 1) * S::SLOTB,
                                 static_cast<const unsigned char*>(in) + (size_t)(lo + j) * B * C * BIN, bytes, bar);
            else
                tma_load_1d(ring + (j & 1) * S::SLOTB,
                            static_cast<const unsigned char*>(in) + (size_t)(lo + j) * B * C * BIN, bytes, bar);
        }
    };
    // fp32 input: the first two raw batches are requested before the taps,
    // the carried rows and the twiddles are loaded, so their latencies
    // overlap (+1 % at C = 512; for 8/16-bit input it measured 0.1-0.2 %
    // slower, so there they are requested after the CTA barrier below)
    constexpr bool EARLY = IN == IN_CF32;
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        *sflag = 0;
        if constexpr (MULTI) fence_proxy_async_smem();   // the slots were last read by the previous range
        if (EARLY) {
            issue(0);
            if (nraw_b > 1) issue(1);
        }
    }

    const float2* tws = args.tw;
    if constexpr (S::TW_SMEM) {
        for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
        tws = tw_s;
    }
    // taps of this pair, shifted so the bucket's zero taps lead: h'[t] = h[t - D]
    unsigned long long h0[TM], h1[TM];
    {
        const float2* taps2 = reinterpret_cast<const float2*>(args.taps);
#pragma unroll
        for (int t = 0; t < TM; ++t) {
            const float2 h = (t >= D) ? __ldg(taps2 + (t - D) * (C / 2) + cp) : make_float2(0.f, 0.f);
            h0[t] = pk2(h.x, h.x);
            h1[t] = pk2(h.y, h.y);
        }
    }
    // carried rows x_i = raw row lo*B - (TM-1) + i, i < TM-1 (zero before the stream)
    float4 carry[TM > 1 ? TM - 1 : 1];
#pragma unroll
    for (int i = 0; i < TM - 1; ++i) {
        const long long r = lo * B - (TM - 1) + i;
        carry[i] = (r >= 0 && r < n_raw) ? load_pair_global<IN>(in, r * C + 2 * cp)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }

    GRP::sync();
    if (!EARLY && tid == 0) {
        issue(0);
        if (nraw_b > 1) issue(1);
    }

    for (long long k = 0; k < nraw_b; ++k) {
        // ------------------------------------------------ wait for slot k
        if (tid == 0) {
            bool ok = rows_of(k) == 0 || mbar_wait_bounded(&bars[k & 1], (uint32_t)((k >> 1) & 1), kWaitLimitNs);
            if (k == 0 && (args.flags & FWD_INJECT_TIMEOUT))     // a barrier nothing arrives on
                ok = ok && mbar_wait_bounded(&bars[2], 0, kInjectedWaitNs);
            if (!ok) {
                // give up: let the copies in flight land, then report
                for (long long j = k; j < k + 2 && j < nraw_b; ++j)
                    if (rows_of(j) > 0) mbar_wait_bounded(&bars[j & 1], (uint32_t)((j >> 1) & 1), kWaitLimitNs);
                atomicExch(args.err, 1);
                *sflag = 1;
            }
        }
        GRP::sync();
        if (*sflag) return false;
        // ---------------------------------------------------------- FIR
        // sequence x_i: i < TM-1 carried rows, then the B rows of slot k.
        // output j = sum_{t < TM} h'[t] x_{j+t}
        {
            const unsigned char* slot = ring + (k & 1) * S::SLOTB + 2 * cp * BIN;
            unsigned long long acc[B][2];
#pragma unroll
            for (int j = 0; j < B; ++j) acc[j][0] = acc[j][1] = 0ull;
            float4 nxt[TM > 1 ? TM - 1 : 1];
#pragma unroll
            for (int i = 0; i < B + TM - 1; ++i) {
                const float4 x = (i < TM - 1) ? carry[i < TM - 1 ? i : 0]
                                              : load_pair_smem<IN>(slot + (size_t)(i - (TM - 1)) * C * BIN);
                const unsigned long long x01 = pk2(x.x, x.y), x23 = pk2(x.z, x.w);
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const int t = i - j;
                    if (t >= 0 && t < TM) {
                        if (IN != IN_CF32 || t >= D) {      // fp32: keep inf/NaN out of unrelated outputs
                            ffma2(acc[j][0], h0[t], x01);
                            ffma2(acc[j][1], h1[t], x23);
                        }
                    }
                }
                if (i >= B) nxt[i - B] = x;
            }
#pragma unroll
            for (int i = 0; i < TM - 1; ++i) carry[i] = nxt[i];
            if constexpr (FIRONLY) {
                const long long sb = (lo + k) * B - (T - 1);
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const long long s = sb + j;
                    if (s >= vlo && s < vhi) {
                        const float2 a = upk2(acc[j][0]), b = upk2(acc[j][1]);
                        __stcs(reinterpret_cast<float4*>(static_cast<float2*>(out) + s * C + 2 * cp),
                               make_float4(a.x, a.y, b.x, b.y));
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const float2 a = upk2(acc[j][0]), b = upk2(acc[j][1]);
                    *reinterpret_cast<float4*>(ybuf + j * S::YSPAN + 2 * cp) = make_float4(a.x, a.y, b.x, b.y);
                }
            }
        }
        GRP::sync();
        // slot k is free: refill it with raw batch k+2
        if (tid == 0 && k + 2 < nraw_b) {
            fence_proxy_async_smem();
            issue(k + 2);
        }
        // ---------------------------------------------------------- FFT
        if constexpr (!FIRONLY) {
            const long long sb = (lo + k) * B - (T - 1);     // output spectrum of batch row 0
            static_for<NST>([&](auto p) {
                fft_stage<C, B, NT, decltype(p)::value, OUT, S::TW_SMEM, S::SPW, false, false, S::LAYOUT, GRP>(
                    ybuf, tws, out, sb, vlo, vhi);
            });
        }
    }
    if constexpr (MULTI) {
        GRP::sync();                                 // every thread is past its last wait
        if (tid == 0)
            for (int i = 0; i < 3; ++i) mbar_inval(&bars[i]);
    }
    return true;
}

template <int C, int TM, int IN, int OUT, bool FIRONLY = false>
__global__ void __launch_bounds__(CarryShape<C, TM, IN>::NT, CarryShape<C, TM, IN>::MINB)
pfb_fwd_carry_kernel(FwdArgs args) {
    using S = CarryShape<C, TM, IN>;
    constexpr int B = S::B, BIN = S::BIN;
    extern __shared__ __align__(128) unsigned char smem[];
    const long long nbt = (args.n_spectra + B - 1) / B;
    const int cps = (int)(gridDim.x / args.n_streams);   // CTAs per stream (the grid is a multiple)
    const int strm = blockIdx.x / cps, bx = blockIdx.x - strm * cps;
    const void* in = static_cast<const unsigned char*>(args.in) + (size_t)strm * args.in_stride * BIN;
    void* out = static_cast<unsigned char*>(args.out) + (size_t)strm * args.out_stride * (OUT == OUT_CF32 ? 8 : 4);
    const long long lo = (long long)bx * nbt / cps;
    const long long hi = (long long)(bx + 1) * nbt / cps;
    carry_range<C, TM, IN, OUT, FIRONLY, CtaGroup, false>(args, in, out, lo, hi, smem);
}

}  // namespace ppf
