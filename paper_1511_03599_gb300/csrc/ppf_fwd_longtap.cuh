// ppf_fwd_longtap.cuh -- fused PFB forward kernel for many taps (T = 17..64).
//
// With many taps the T-1 halo rows a batch of output spectra shares with the
// previous batch (the overlap of neighbouring blocks, Sec. 3.2) no longer fit
// in registers, and for 32-bit input not in shared memory either (63 rows of
// 4 KB at C = 512).  So each batch of B = 16 output spectra streams all
// B + T - 1 raw rows it needs through a 3-slot TMA ring in chunks of RC rows:
// the rows new to the batch come from HBM, the halo rows from L2, where the
// previous batches of the same CTA just brought them (each raw sample is read
// from HBM once; L2 -> SM traffic is (B + T - 1) / B times the input).
//
// FIR (Alg. 1), per thread = one channel pair, taps outermost: a window of B
// rows lives in registers; tap t adds h[t] * x[j + t] to output j for all B
// outputs, then the dead row t is replaced by row t + B (slot (j + t) mod B
// holds row j + t).  Each row is loaded and converted once per batch, each
// tap loaded once per batch (from L1/L2), and every FMA is a packed
// (re, im) x (h, h) pair.  Chunks are consumed in order: every thread waits
// for a chunk's TMA barrier itself, and each warp arrives on the chunk
// slot's "empty" barrier when it is done, so thread 0 refills a slot without
// a CTA-wide barrier.  The filtered batch then goes through the same
// warp-local DFT stages (Eq. 2) as the carry kernel.
#pragma once

#include "ppf_fwd_carry.cuh"

#ifndef PPF_LONGTAP_STAGE
#define PPF_LONGTAP_STAGE 1
#endif

namespace ppf {

template <int C, int IN>
struct LongShape {
    static constexpr int NT = C / 2;                                 // one channel pair per thread
    static constexpr int B = 16;                                     // output spectra per batch
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr int RC = BIN <= 4 ? 16 : 8;                     // rows per ring chunk
    static constexpr int NS = 3;                                     // ring slots
    static constexpr int NWARP = NT / 32;
    static constexpr int SPW = B / (NWARP > 0 ? NWARP : 1);          // spectra per warp in the DFT
    static constexpr int YBYTES = B * C * 8;
    static constexpr int TWBYTES = tw_size(C) * 8;
    static constexpr int CHUNKB = RC * C * BIN;
    static constexpr int RING_OFF = YBYTES + TWBYTES;
    static constexpr int BAR_OFF = RING_OFF + NS * CHUNKB;           // NS full + NS empty + 1 + flag
    // STAGE: each thread's taps stream through TD shared-memory slots of its
    // own (cp.async, TD taps ahead) instead of a rolling set of registers --
    // where it measured faster: C = 512 with int16 (+3 .. +10 %) or fp32 input
    // (+12 .. +13 %); for int8 at C = 512 (-6 % at T = 17, 32; +4 % at T = 64)
    // and at C = 256 (-8 .. -13 %) the registers stay
    static constexpr bool STAGE = PPF_LONGTAP_STAGE != 0 && C == 512 && IN != IN_CI8;
    static constexpr int TD = 8;
    static constexpr int TAP_OFF = BAR_OFF + 8 * (2 * NS + 2);
    static constexpr int SMEM = TAP_OFF + (STAGE ? TD * NT * 8 : 0);
    static constexpr bool OK = C >= 64 && C <= 512 && NT % 32 == 0 && SPW >= 1 && SPW * NWARP == B &&
                               warp_fft_ok(C, SPW) && SMEM <= 226 * 1024 && B % RC == 0;
};

template <int C, int IN, int OUT>
__global__ void __launch_bounds__(LongShape<C, IN>::NT, 1) pfb_fwd_longtap_kernel(FwdArgs args) {
    using S = LongShape<C, IN>;
    constexpr int NT = S::NT, B = S::B, BIN = S::BIN, RC = S::RC, NS = S::NS, NWARP = S::NWARP;
    constexpr int NST = fft_stages(C);
    constexpr int OB = OUT == OUT_CF32 ? 8 : 4;
    static_assert(S::OK, "shape not supported by the long-tap kernel");
    static_assert(!S::STAGE || B % S::TD == 0, "a tap's staging slot is its index in the block mod TD");
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ybuf = reinterpret_cast<float2*>(smem);
    float2* tw_s = reinterpret_cast<float2*>(smem + S::YBYTES);
    unsigned char* ring = smem + S::RING_OFF;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);    // [NS] chunk landed
    uint64_t* empty = full + NS;                                         // [NS] every warp is done with it
    uint64_t* inj = full + 2 * NS;                                       // never completed (testing aid)
    volatile int* sdead = reinterpret_cast<volatile int*>(full + 2 * NS + 1);
    float2* stap = reinterpret_cast<float2*>(smem + S::TAP_OFF);          // [TD][NT] staged taps (STAGE)

    const int tid = threadIdx.x, lane = tid & 31;
    const int cp = tid;
    const long long n_spectra = args.n_spectra;
    const int T = args.T;                        // 17 .. 64
    const long long n_raw = n_spectra + T - 1;
    const long long nbt = (n_spectra + B - 1) / B;
    const int nch = (B + T - 1 + RC - 1) / RC;   // chunks per batch
    const float2* taps2 = reinterpret_cast<const float2*>(args.taps);   // [t][pair]

    for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NWARP);
        }
        mbar_init(inj, 1);
        fence_mbar_init();
        *sdead = 0;
    }
    __syncthreads();

    // Chunk uses are counted over the whole kernel (g), so slots and barrier
    // phases run on across the stream segments of the CTA's share.
    long long g_base = 0;           // first chunk use of the current segment
    long long issued = 0;           // thread 0: chunk uses issued so far (over the kernel)
    long long seg_end = 0;          // chunk uses up to the end of the current segment
    const unsigned char* seg_in = nullptr;
    long long seg_lo = 0;
    auto chunk_rows = [&](long long rel) -> long long {   // rows of chunk `rel` of the segment
        const long long k = rel / nch, c = rel % nch;
        const long long r0 = (seg_lo + k) * B + c * RC;
        long long rows = n_raw - r0;
        rows = rows < RC ? rows : RC;
        const long long need = B + T - 1 - c * RC;        // rows of the batch in this chunk
        rows = rows < need ? rows : need;
        return rows < 0 ? 0 : rows;
    };
    auto issue = [&](long long g) {             // thread 0: chunk use g (of the current segment)
        const long long rel = g - g_base;
        const int s = (int)(g % NS);
        const long long rows = chunk_rows(rel);
        mbar_expect_tx(&full[s], (uint32_t)(rows * C * BIN));
        if (rows > 0) {
            const long long k = rel / nch, c = rel % nch;
            const long long r0 = (seg_lo + k) * B + c * RC;
            tma_load_1d(ring + s * S::CHUNKB, seg_in + (size_t)r0 * C * BIN, (uint32_t)(rows * C * BIN), &full[s]);
        }
    };
    // thread 0: refill every slot whose previous use all warps have released
    auto refill = [&](long long upto) {
        for (; issued < upto && issued < seg_end; ++issued) {
            if (issued >= NS) {
                const long long prev = issued - NS;
                if (!mbar_wait_bounded(&empty[prev % NS], (uint32_t)((prev / NS) & 1), kWaitLimitNs)) {
                    atomicExch(args.err, 1);
                    *sdead = 1;
                    return;
                }
            }
            fence_proxy_async_smem();
            issue(issued);
        }
    };
    // every thread: the chunk in `slot` (phase parity `par`) has landed
    auto wait_full = [&](int slot, int par) {
        if (*sdead) return;
        if (!mbar_wait_bounded(&full[slot], (uint32_t)par, kWaitLimitNs)) {
            atomicExch(args.err, 1);
            *sdead = 1;
        }
    };
    auto release = [&](int slot) {              // every thread: done with the chunk in `slot`
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(&empty[slot]);
    };

    // STAGE: tap t of the pair goes to the thread's slot t mod TD; one commit
    // group per tap (an empty group past the last tap), so a wait for all
    // but the TD-1 youngest groups means "tap t has landed"
    const float2* tp = taps2 + cp;
    auto stage_tap = [&](int t) {
        if constexpr (S::STAGE) {
            if (t < T) cp_async<8>(&stap[(t % S::TD) * NT + tid], tp + (size_t)t * (C / 2));
            cp_async_commit();
        }
    };
    BatchShare share(nbt, args.n_streams, blockIdx.x, gridDim.x);
    long long strm, lo, hi;
    bool first = true;
    while (share.next(strm, lo, hi)) {
        seg_in = static_cast<const unsigned char*>(args.in) + (size_t)strm * args.in_stride * BIN;
        void* out = static_cast<unsigned char*>(args.out) + (size_t)strm * args.out_stride * OB;
        seg_lo = lo;
        seg_end = g_base + (hi - lo) * nch;
        if (tid == 0) {
            if (first && (args.flags & FWD_INJECT_TIMEOUT) && !mbar_wait_bounded(inj, 0, kInjectedWaitNs)) {
                atomicExch(args.err, 1);
                *sdead = 1;
            }
            if (!*sdead) refill(g_base + NS);
        }
        first = false;
        __syncthreads();

#pragma unroll
        for (int t = 0; t < S::TD; ++t) stage_tap(t);                 // the first batch's first taps
        for (long long k = lo; k < hi; ++k) {
            const long long g0 = g_base + (k - lo) * nch;      // first chunk use of this batch
            const int s0 = (int)(g0 % NS), q0 = (int)((g0 / NS) & 1);
            // slot and phase parity of chunk c of this batch (chunk use g0 + c)
            auto slot_of = [&](int c) { return (s0 + c) % NS; };
            auto par_of = [&](int c) { return (q0 + (s0 + c) / NS) & 1; };
            // ------------------------------------------------------------- FIR
            // channel-paired accumulators: acc[j][0] = (re, re), acc[j][1] = (im, im) of
            // channels (2cp, 2cp+1) for output j; window rows likewise as (re, re), (im, im)
            // pairs, and each tap is used as loaded, (h[2cp], h[2cp+1])
            unsigned long long acc[B][2];
#pragma unroll
            for (int j = 0; j < B; ++j) acc[j][0] = acc[j][1] = 0ull;
            unsigned long long xr[B], xi[B];
            auto load_row = [&](const unsigned char* p, int i) {
                const float4 v = load_pair_smem<IN>(p);
                xr[i] = pk2(v.x, v.z);
                xi[i] = pk2(v.y, v.w);
            };
            // rows 0 .. B-1 of the batch fill the window (B / RC whole chunks)
#pragma unroll
            for (int c = 0; c < B / RC; ++c) {
                const int sl = slot_of(c);
                wait_full(sl, par_of(c));
                const unsigned char* src = ring + sl * S::CHUNKB + 2 * cp * BIN;
#pragma unroll
                for (int i = 0; i < RC; ++i) load_row(src + (size_t)i * C * BIN, c * RC + i);
                release(sl);
                if (tid == 0 && !*sdead) refill(g0 + c + 1 + NS);
            }
            // without STAGE: taps 4 ahead in a rolling set of registers (tap t lives in
            // hq[t % 4]); the plan pads the tap table with zero rows, so loads past T
            // stay in bounds
            unsigned long long hq[4];
            if constexpr (!S::STAGE) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 h = __ldg(tp + i * (C / 2));
                    hq[i] = pk2(h.x, h.y);
                }
            }
            // taps in blocks of B: tap t = tb + u uses window slot (j + u) mod B for output j,
            // then slot u takes row t + B, in chunk (t + B) / RC, at row (t + B) mod RC = u mod RC.
            // FULL: every tap of the block exists and every row it loads lies in the batch
            // (tb + B <= T - 1), so the block runs without per-tap checks.
            auto block = [&](int tb, auto full_tag) {
                constexpr bool FULL = decltype(full_tag)::value != 0;
                int csl[B / RC];
                const unsigned char* csrc[B / RC];
#pragma unroll
                for (int h = 0; h < B / RC; ++h) {
                    const int c = (tb + B) / RC + h;
                    csl[h] = slot_of(c);
                    csrc[h] = ring + csl[h] * S::CHUNKB + 2 * cp * BIN;
                    if (FULL || tb + h * RC < T - 1) wait_full(csl[h], par_of(c));
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int t = tb + u;
                    if (FULL || t < T) {
                        unsigned long long h;
                        if constexpr (S::STAGE) {
                            cp_async_wait<S::TD - 1>();              // tap t has landed
                            const float2 hv = stap[(u % S::TD) * NT + tid];   // t mod TD (tb is a multiple of B)
                            h = pk2(hv.x, hv.y);
                            stage_tap(t + S::TD);
                        } else {
                            h = hq[u % 4];
                            const float2 hn = __ldg(tp + (t + 4) * (C / 2));
                            hq[u % 4] = pk2(hn.x, hn.y);
                        }
#pragma unroll
                        for (int j = 0; j < B; ++j) {
                            ffma2(acc[j][0], h, xr[(j + u) % B]);
                            ffma2(acc[j][1], h, xi[(j + u) % B]);
                        }
                        if (FULL || t < T - 1) {                // row t + B exists in the batch
                            load_row(csrc[u / RC] + (size_t)(u % RC) * C * BIN, u);
                            if (u % RC == RC - 1 || (!FULL && t == T - 2)) {
                                release(csl[u / RC]);
                                if (tid == 0 && !*sdead) refill(g0 + (tb + B) / RC + u / RC + 1 + NS);
                            }
                        }
                    }
                }
            };
            int tb = 0;
            for (; tb + B <= T - 1; tb += B) block(tb, ic<1>{});
            for (; tb < T; tb += B) block(tb, ic<0>{});
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const float2 r = upk2(acc[j][0]), im = upk2(acc[j][1]);
                *reinterpret_cast<float4*>(ybuf + j * C + 2 * cp) = make_float4(r.x, im.x, r.y, im.y);
            }
            if (k + 1 < hi) {                                        // the next batch's first taps land
#pragma unroll                                                       // during this batch's DFT
                for (int t = 0; t < S::TD; ++t) stage_tap(t);
            }
            __syncthreads();
            // ------------------------------------------------------------- FFT
            const long long vhi = *sdead ? 0 : n_spectra;           // a CTA that gave up stores nothing
            static_for<NST>([&](auto p) {
                fft_stage<C, B, NT, decltype(p)::value, OUT, true, S::SPW>(ybuf, tw_s, out, k * B, 0, vhi);
            });
            __syncthreads();   // every warp is done with ybuf before the next FIR writes it
        }
        g_base = seg_end;
    }
    // leave only after every copy this CTA issued has landed
    if constexpr (S::STAGE) cp_async_wait<0>();
    if (tid == 0)
        for (long long g = (issued > NS ? issued - NS : 0); g < issued; ++g)
            mbar_wait_bounded(&full[g % NS], (uint32_t)((g / NS) & 1), kWaitLimitNs);
}

}  // namespace ppf
