// ppf_fwd_cluster.cuh -- fused PFB forward kernel for large channel counts
// on a thread-block cluster (used where it measured faster than the
// single-CTA kernels: fp32 input at C = 768 and 2048).
//
// The FIR state of a C-channel stream (T-1 carried rows per channel) does not
// fit one SM at these sizes, so a cluster of Q = C/KS CTAs shares a stream
// (KS = 256 channels per CTA, two CTAs per SM, up to C = 2048; KS = 512 for
// the larger C, keeping the cluster within the portable size of 8):
//   * CTA q owns channels [KS*q, KS*q + KS) for the FIR (Alg. 1): each of its
//     KS threads keeps one channel with the T-1 halo rows carried in
//     registers; raw rows arrive by TMA bulk copies of the CTA's slice of
//     each spectrum into a double-buffered ring; the filtered slice goes to
//     one of two slice buffers (batch parity);
//   * CTA q transforms spectra [q*SPC, (q+1)*SPC) of each batch (Eq. 2): the
//     first DFT stage gathers its columns from all Q CTAs' slice buffers
//     through distributed shared memory (plain loads from the cluster's
//     shared-memory window, no multicast) into the CTA's stage buffer; the
//     remaining stages run there and the last one stores the spectra.
// The loop is software-pipelined by one batch with ONE cluster barrier per
// batch, split into arrive and wait: iteration k filters batch k into slice
// buffer k&1, runs the middle DFT stages of batch k-1, arrives, runs the
// last stage of batch k-1, waits, and gathers batch k.  The barrier of iteration k publishes the slices of batch
// k and certifies that every gather of batch k-1 is done, so the slice buffer
// that batch k+1 overwrites is no longer read by anyone.  A last barrier after
// the loop keeps every CTA resident until no peer reads its shared memory.
// Every raw sample is read from HBM once and y never leaves the cluster.
// Every CTA reaches every cluster barrier: a CTA whose bounded wait gives up
// records the error, stops issuing and waiting for copies and storing output,
// and keeps taking part in the barriers until the loop ends.
#pragma once

#include "ppf_fwd.cuh"

// Where the generic kernel measured faster, the cluster kernel is not used:
// for 8/16-bit input at C = 2048 (int8 T=8: 265 GS/s with 8-spectrum batches
// vs 202; int16 T=8: 212 vs 170) and at C = 4096 (int16 T=8, a ring of HS + 1
// slots beside 2-spectrum batches: 173 vs 113; fp32 T=8, 4-spectrum batches
// loaded directly: 117 vs 104, T=4: 144 vs 116).  fp32 input at C = 2048
// keeps it (T=8: 158 vs 145 GS/s), and so does fp32 input at C = 768 (T=8:
// 139 vs 109), where 8/16-bit input now runs faster on the generic kernel's
// ring (int8 T=16: 142 vs 116; int16 T=8: 167 vs 154).  The switches below
// restore it elsewhere.
#ifndef PPF_CLUSTER_2048
#define PPF_CLUSTER_2048 0
#endif
#ifndef PPF_CLUSTER_CF32
#define PPF_CLUSTER_CF32 1       // fp32 input at C = 2048
#endif
#ifndef PPF_CLUSTER_4096
#define PPF_CLUSTER_4096 0       // fp32 input and 5-8-tap int16 input at C = 4096
#endif
#ifndef PPF_CLUSTER_768
#define PPF_CLUSTER_768 1        // fp32 input at C = 768
#endif

namespace ppf {

// channels per CTA of a cluster: 256 (two CTAs per SM) where the cluster
// stays within the portable size of 8, else 512
constexpr int cluster_slice(int C) { return C / 256 <= 8 ? 256 : 512; }

template <int C, int KS, int BIN, int B>
constexpr int cluster_smem(bool tw_smem) {
    return 3 * B * KS * 8 + 2 * B * KS * BIN + (tw_smem ? tw_size(C) * 8 : 0) + 64;
}
template <int C, int TM, int IN>
struct ClusterShape {
    static constexpr int KS = cluster_slice(C);                      // channels per CTA
    static constexpr int Q = C >= KS ? C / KS : 1;                   // CTAs per cluster
    static constexpr int NT = KS;                                    // one channel per thread
    static constexpr int MINB = KS == 256 ? 2 : 1;                   // CTAs per SM
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr int CAP = KS == 256 ? 112 * 1024 + 64 : 226 * 1024;
    static constexpr int B0 = IN == IN_CI8 ? 16 : 8;
    static constexpr int BUP = Q * ((B0 + Q - 1) / Q);
    static constexpr int BDN = Q * (B0 / Q > 0 ? B0 / Q : 1);
    static constexpr int B = cluster_smem<C, KS, BIN, BUP>(false) <= CAP ? BUP : BDN;   // spectra per batch
    static constexpr int SPC = B / Q;                                // spectra each CTA transforms
    static constexpr int YLB = B * KS * 8;                           // one slice buffer == stage buffer
    static constexpr int SLOTB = B * KS * BIN;                       // raw rows of the slice
    static constexpr bool TW_SMEM = cluster_smem<C, KS, BIN, B>(true) <= CAP;
    static constexpr int WK_OFF = 2 * YLB;
    static constexpr int TW_OFF = 3 * YLB;
    static constexpr int RING_OFF = TW_OFF + (TW_SMEM ? tw_size(C) * 8 : 0);
    static constexpr int SMEM = RING_OFF + 2 * SLOTB + 64;
    // where it measured faster than the single-CTA kernels: fp32 input at
    // C = 768 and 2048 (the generic kernel won at C = 1024, 1536, 3072 and
    // 4096, and for 8/16-bit input at C = 768 and 2048)
    static constexpr bool WANTED = (C == 2048 && ((IN == IN_CF32 && PPF_CLUSTER_CF32) || PPF_CLUSTER_2048)) ||
                                   (C == 768 && PPF_CLUSTER_768 && IN == IN_CF32) ||
                                   (C == 4096 && PPF_CLUSTER_4096 && (IN == IN_CF32 || (IN == IN_CI16 && TM == 8)));
    static constexpr bool OK = WANTED && C % KS == 0 && Q >= 2 && Q <= 8 && TM <= 16 && B >= TM - 1 &&
                               SPC * C == B * KS && SMEM <= CAP;
};

// Split cluster barrier: arrive (release: this thread's earlier writes, e.g.
// of its slice buffer, become visible to the cluster) and wait (acquire).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster
// (32-bit shared::cluster window).
__device__ __forceinline__ uint32_t dsmem_map(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 dsmem_ld_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// First DFT stage of the CTA's SPC spectra: gather the columns from the
// filtered slices of all CTAs of the cluster (rb[r]: shared::cluster address
// of CTA r's slice; local: shared::cta address of this CTA's own slice, the
// address `mapa` maps to another rank), radix-R DFT, inter-stage twiddles.
// Results stay in v.
template <int C, int KS, int SPC, int NT, int Q, int IPT>
__device__ __forceinline__ void cluster_stage0_load(const uint32_t (&rb)[Q], uint32_t local,
                                                    float2 (&v)[IPT][fft_radix(C, 0)],
                                                    const float2* __restrict__ tws, bool tw_smem, int q) {
    constexpr int R = fft_radix(C, 0);
    constexpr int NN = C / R;                  // N_1
    constexpr int TOTAL = SPC * NN;
    const int tid = threadIdx.x;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = tid + it * NT;
        if (item >= TOTAL) break;
        const int sp = item / NN, b = item % NN;
        const uint32_t row = (uint32_t)(q * SPC + sp) * (KS * 8);       // batch row of the spectrum
#pragma unroll
        for (int a = 0; a < R; ++a) {
            if constexpr (KS % NN == 0) {      // column a lies in one slice for every b
                constexpr int PER = KS / NN;
                v[it][a] = dsmem_ld_f2(rb[a / PER] + row + (uint32_t)(((a % PER) * NN + b) * 8));
            } else {                           // the slice depends on b
                const int c = NN * a + b;
                v[it][a] = dsmem_ld_f2(dsmem_map(local + row + (uint32_t)((c % KS) * 8), (uint32_t)(c / KS)));
            }
        }
    }
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = tid + it * NT;
        if (item >= TOTAL) break;
        const int b = item % NN;
        dft_reg<R>(v[it]);
        if (tw_smem) apply_twiddles<R, NN, true>(v[it], tws, b);
        else apply_twiddles<R, NN, false>(v[it], tws, b);
    }
}
template <int C, int SPC, int NT, int IPT>
__device__ __forceinline__ void cluster_stage0_store(const float2 (&v)[IPT][fft_radix(C, 0)], float2* __restrict__ work) {
    constexpr int R = fft_radix(C, 0);
    constexpr int NN = C / R;
    constexpr int TOTAL = SPC * NN;
    const int tid = threadIdx.x;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = tid + it * NT;
        if (item >= TOTAL) break;
        const int sp = item / NN, b = item % NN;
        float2* dst = work + sp * C;
#pragma unroll
        for (int k = 0; k < R; ++k) dst[phys<C, 1>(k * NN + b)] = v[it][k];
    }
}

template <int C, int TM, int IN, int OUT>
__global__ void __cluster_dims__(ClusterShape<C, TM, IN>::Q, 1, 1) __launch_bounds__(ClusterShape<C, TM, IN>::NT, ClusterShape<C, TM, IN>::MINB)
pfb_fwd_cluster_kernel(FwdArgs args) {
    using S = ClusterShape<C, TM, IN>;
    constexpr int NT = S::NT, B = S::B, BIN = S::BIN, Q = S::Q, SPC = S::SPC, kSlice = S::KS;
    constexpr int NST = fft_stages(C);
    static_assert(NST >= 2, "the pipelined loop runs the middle stages before the barrier and the last after it");
    constexpr int R0 = fft_radix(C, 0);
    constexpr int IPT0 = (SPC * (C / R0) + NT - 1) / NT;
    constexpr int OB = OUT == OUT_CF32 ? 8 : 4;
    static_assert(S::OK, "shape not supported by the cluster kernel");
    extern __shared__ __align__(128) unsigned char smem[];
    float2* ylb = reinterpret_cast<float2*>(smem);                         // two slice buffers
    float2* wk = reinterpret_cast<float2*>(smem + S::WK_OFF);              // stage buffer
    float2* tw_s = reinterpret_cast<float2*>(smem + S::TW_OFF);
    unsigned char* ring = smem + S::RING_OFF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + 2 * S::SLOTB);     // 3 barriers
    volatile int* sdead = reinterpret_cast<int*>(bars + 3);                // this CTA gave up

    const int tid = threadIdx.x;
    const int q = (int)cluster_rank();               // slice of this CTA
    const long long n_spectra = args.n_spectra;
    const int T = args.T;
    const int D = TM - T;
    const long long n_raw = n_spectra + T - 1;
    const long long nbt = (n_spectra + B - 1) / B;

    const float2* tws = args.tw;
    if constexpr (S::TW_SMEM) {
        for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
        tws = tw_s;
    }
    unsigned long long h[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) {
        const float x = (t >= D) ? __ldg(args.taps + (t - D) * C + q * kSlice + tid) : 0.f;
        h[t] = pk2(x, x);
    }
    uint32_t rb[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) rb[r] = dsmem_map(smem_addr(ylb), (uint32_t)r);
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        *sdead = 0;
    }
    __syncthreads();

    // The cluster's share of the batches of all streams (the same for every
    // CTA of the cluster), walked as single-stream segments.  kb counts the
    // raw batches of earlier segments: raw batch k of a segment is use kb + k
    // of the ring slot (kb + k) & 1 and of the slice buffer (kb + k) & 1;
    // every ring use completes one phase of its slot's barrier (zero bytes
    // when it has no rows), so slots, phases and slice buffers run on across
    // segments.
    BatchShare share(nbt, args.n_streams, blockIdx.x / Q, gridDim.x / Q);
    long long strm, lo, hi, kb = 0;
    while (share.next(strm, lo, hi)) {
        const unsigned char* in = static_cast<const unsigned char*>(args.in) + (size_t)strm * args.in_stride * BIN;
        void* out = static_cast<unsigned char*>(args.out) + (size_t)strm * args.out_stride * OB;
        const long long nb = hi - lo;
        const long long vlo = lo * B, vhi = (hi * B < n_spectra) ? hi * B : n_spectra;
        const long long nraw_b = (T > 1) ? nb + 1 : nb;

        float2 carry[TM > 1 ? TM - 1 : 1];
#pragma unroll
        for (int i = 0; i < TM - 1; ++i) {
            const long long r = lo * B - (TM - 1) + i;
            carry[i] = (r >= 0 && r < n_raw) ? load_one_global<IN>(in, r * C + q * kSlice + tid)
                                             : make_float2(0.f, 0.f);
        }
        auto rows_of = [&](long long j) -> long long {
            const long long r = n_raw - (lo + j) * B;
            return r <= 0 ? 0 : (r < B ? r : B);
        };
        // raw batch j: the CTA's slice of rows [(lo+j)B, (lo+j)B + B), one bulk copy per row
        auto issue = [&](long long j) {
            const long long rows = rows_of(j);
            const long long u = kb + j;
            uint64_t* bar = &bars[u & 1];
            mbar_expect_tx(bar, (uint32_t)(rows * kSlice * BIN));
            unsigned char* dst = ring + (u & 1) * S::SLOTB;
            const unsigned char* src = in + ((size_t)(lo + j) * B * C + (size_t)q * kSlice) * BIN;
            for (long long r = 0; r < rows; ++r)
                tma_load_1d(dst + r * kSlice * BIN, src + (size_t)r * C * BIN, kSlice * BIN, bar);
        };
        auto wait_use = [&](long long j, uint64_t limit) -> bool {
            const long long u = kb + j;
            return mbar_wait_bounded(&bars[u & 1], (uint32_t)((u >> 1) & 1), limit);
        };
        if (tid == 0 && !*sdead) {
            fence_proxy_async_smem();   // the slots were last read by an earlier segment's FIR
            issue(0);
            if (nraw_b > 1) issue(1);
        }

        // iteration k: FIR of batch k (k < nraw_b), later stages of batch k-1 (k >= 1)
        for (long long k = 0; k <= nraw_b; ++k) {
            const bool fir = k < nraw_b;
            if (!fir) __syncthreads();   // the gathered batch is complete in wk
            if (fir) {
                // ------------------------------------------------ wait for slot k
                if (tid == 0 && !*sdead) {
                    bool ok = wait_use(k, kWaitLimitNs);
                    if (kb == 0 && k == 0 && (args.flags & FWD_INJECT_TIMEOUT))
                        ok = ok && mbar_wait_bounded(&bars[2], 0, kInjectedWaitNs);
                    if (!ok) {
                        for (long long j = k; j < k + 2 && j < nraw_b; ++j) wait_use(j, kWaitLimitNs);
                        atomicExch(args.err, 1);
                        *sdead = 1;
                    }
                }
                __syncthreads();
                const bool dead = *sdead != 0;
                // ------------------------------------------------------ FIR
                unsigned long long acc[B];
                if (!dead) {
                    const unsigned char* slot = ring + ((kb + k) & 1) * S::SLOTB + tid * BIN;
#pragma unroll
                    for (int j = 0; j < B; ++j) acc[j] = 0ull;
                    float2 nxt[TM > 1 ? TM - 1 : 1];
#pragma unroll
                    for (int i = 0; i < B + TM - 1; ++i) {
                        const float2 x = (i < TM - 1) ? carry[i < TM - 1 ? i : 0]
                                                      : load_one_smem<IN>(slot + (size_t)(i - (TM - 1)) * kSlice * BIN);
                        const unsigned long long xx = pk2(x.x, x.y);
#pragma unroll
                        for (int j = 0; j < B; ++j) {
                            const int t = i - j;
                            if (t >= 0 && t < TM) {
                                if (IN != IN_CF32 || t >= D) ffma2(acc[j], h[t], xx);
                            }
                        }
                        if (i >= B) nxt[i - B] = x;
                    }
#pragma unroll
                    for (int i = 0; i < TM - 1; ++i) carry[i] = nxt[i];
                }
                __syncthreads();
                if (tid == 0 && !dead && k + 2 < nraw_b) {   // slot k is free: refill it
                    fence_proxy_async_smem();
                    issue(k + 2);
                }
                if (!dead) {
                    float2* yl = ylb + ((kb + k) & 1) * (B * kSlice);
#pragma unroll
                    for (int j = 0; j < B; ++j) yl[j * kSlice + tid] = upk2(acc[j]);
                }
            }
            const long long sbp = (lo + k - 1) * B - (T - 1) + q * SPC;   // first output spectrum of batch k-1
            const long long pvlo = *sdead ? vhi : vlo;                      // a CTA that gave up stores nothing
            if (k >= 1) {                  // middle DFT stages of batch k-1
                static_for<NST - 2>([&](auto pm1) {
                    fft_stage<C, SPC, NT, decltype(pm1)::value + 1, OUT, S::TW_SMEM>(wk, tws, out, sbp, pvlo, vhi);
                });
            }
            if (fir) cluster_arrive();     // slices of batch k written; gathers of batch k-1 done
            if (k >= 1) fft_stage<C, SPC, NT, NST - 1, OUT, S::TW_SMEM>(wk, tws, out, sbp, pvlo, vhi);
            if (fir) {
                cluster_wait();
                float2 v[IPT0][R0];
                const uint32_t off = (uint32_t)(((kb + k) & 1) * (B * kSlice * 8));
                uint32_t rbk[Q];
#pragma unroll
                for (int r = 0; r < Q; ++r) rbk[r] = rb[r] + off;
                cluster_stage0_load<C, kSlice, SPC, NT, Q, IPT0>(rbk, smem_addr(ylb) + off, v, tws, S::TW_SMEM, q);
                cluster_stage0_store<C, SPC, NT, IPT0>(v, wk);   // stage 2 of batch k-1 has read wk
            }
            // (the next iteration's first CTA barrier orders these writes before stage 1)
        }
        kb += nraw_b;
    }
    cluster_arrive();   // no CTA leaves while a peer may still gather from it
    cluster_wait();
}

}  // namespace ppf
