// ppf_fwd_push.cuh -- fused PFB forward kernel for large channel counts on a
// thread-block cluster whose CTAs PUSH their filtered channels to the CTA
// that transforms each spectrum (C = 2048 and 4096).
//
// A C-channel stream's FIR state (T-1 carried rows per channel) does not fit
// one SM at these sizes, so a cluster of Q CTAs shares each stream:
//   * FIR (Alg. 1): CTA q owns channels [q*KS, q*KS + KS), one per thread,
//     with the T-1 halo rows carried in registers between batches; raw rows
//     of its slice arrive by TMA bulk copies into a double-buffered ring.
//   * Exchange: spectrum j of a batch of B belongs to CTA j / SPC (SPC = B/Q
//     spectra per CTA).  Each thread stores its filtered value of spectrum j
//     straight into that CTA's receive buffer with st.async (an asynchronous
//     store to distributed shared memory that completes bytes on the
//     receiver's "full" mbarrier): one store per filtered sample, no
//     cluster-wide barrier, no gather loads.
//   * DFT (Eq. 2): each CTA transforms its SPC spectra in its receive buffer
//     (CTA-wide in-place stages, then coalesced streaming stores).
// Flow control is point to point: receive buffers are double-buffered by
// batch parity; a CTA refills receiver r's buffer b only after r has arrived
// (remote mbarrier arrive) on the sender's "empty" barrier b, i.e. after r
// transformed the batch that last used it.  The loop is pipelined by one
// batch: iteration k filters and pushes batch k, then transforms batch k-1.
// Every raw sample is read from HBM once; y never leaves the cluster.
//
// Every wait is bounded.  A CTA whose wait gives up lets its own copies in
// flight land, records the error and stops copying, pushing and storing; its
// peers' waits on it then run out too.  Every CTA still reaches the final
// cluster barrier, so none exits while a peer may write to its shared memory.
#pragma once

#include "ppf_fwd_cluster.cuh"

namespace ppf {

// Launch shape of the push kernel (complex int8 input; the other input types
// keep the kernels of the earlier selection at these sizes).
template <int C, int TM, int IN>
struct PushShape {
    static constexpr int Q = C == 4096 ? 8 : 4;                      // CTAs per cluster
    static constexpr int KS = C / Q;                                 // channels per CTA (FIR slice)
    static constexpr int NT = KS;                                    // one channel per thread
    static constexpr int B = 16;                                     // spectra per batch
    static constexpr int SPC = B / Q;                                // spectra each CTA transforms
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr int RBUF = SPC * C * 8;                         // one receive buffer
    static constexpr int TWBYTES = tw_size(C) * 8;
    static constexpr int SLOTB = B * KS * BIN;                       // raw rows of the slice
    static constexpr int TW_OFF = 2 * RBUF;
    static constexpr int RING_OFF = TW_OFF + TWBYTES;
    static constexpr int BAR_OFF = RING_OFF + 2 * SLOTB;             // 7 barriers + flag
    static constexpr int SMEM = BAR_OFF + 64;
    static constexpr int MINB = 1;
    static constexpr bool OK = (C == 2048 || C == 4096) && IN == IN_CI8 && TM <= 16 && B >= TM - 1 &&
                               SPC * Q == B && SMEM <= 226 * 1024 && fft_items_fit(C, SPC, NT);
};

// Asynchronous 8-byte store into another CTA's shared memory, completing 8
// bytes of transaction count on that CTA's mbarrier `rbar` (both addresses in
// the shared::cluster window).
__device__ __forceinline__ void st_async_f2(uint32_t raddr, float2 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.x), "f"(v.y), "r"(rbar)
                 : "memory");
}
// Arrive (release at cluster scope) on an mbarrier of another CTA.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t rbar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}
// Local arrival that also expects `bytes` more of transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// try_wait with acquire at cluster scope: the data other CTAs wrote before
// completing the phase is visible after it returns true.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int C, int TM, int IN, int OUT>
__global__ void __cluster_dims__(PushShape<C, TM, IN>::Q, 1, 1) __launch_bounds__(PushShape<C, TM, IN>::NT, 1)
pfb_fwd_push_kernel(FwdArgs args) {
    using S = PushShape<C, TM, IN>;
    constexpr int NT = S::NT, B = S::B, BIN = S::BIN, Q = S::Q, SPC = S::SPC, KS = S::KS;
    constexpr int NST = fft_stages(C);
    constexpr int OB = OUT == OUT_CF32 ? 8 : 4;
    static_assert(S::OK, "shape not supported by the push kernel");
    extern __shared__ __align__(128) unsigned char smem[];
    float2* rbuf = reinterpret_cast<float2*>(smem);                         // [2][SPC][C]
    float2* tw_s = reinterpret_cast<float2*>(smem + S::TW_OFF);
    unsigned char* ring = smem + S::RING_OFF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
    uint64_t* raw_bar = bars;            // [2] TMA copies of raw slots
    uint64_t* inj_bar = bars + 2;        // never completed (testing aid)
    uint64_t* full_bar = bars + 3;       // [2] receive buffer b holds its batch
    uint64_t* empty_bar = bars + 5;      // [2] every receiver is done with its buffer b
    volatile int* sdead = reinterpret_cast<volatile int*>(bars + 7);

    const int tid = threadIdx.x;
    const int q = (int)cluster_rank();
    const long long n_spectra = args.n_spectra;
    const int T = args.T;
    const int D = TM - T;
    const long long n_raw = n_spectra + T - 1;
    const long long nbt = (n_spectra + B - 1) / B;
    constexpr uint32_t kRecvBytes = (uint32_t)SPC * C * 8;   // bytes each receiver gets per batch

    for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
    unsigned long long h[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) {
        const float x = (t >= D) ? __ldg(args.taps + (t - D) * C + q * KS + tid) : 0.f;
        h[t] = pk2(x, x);
    }
    if (tid == 0) {
        mbar_init(&raw_bar[0], 1);
        mbar_init(&raw_bar[1], 1);
        mbar_init(inj_bar, 1);
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], Q);
        mbar_init(&empty_bar[1], Q);
        fence_mbar_init();
        *sdead = 0;
        // the receive buffers expect the first two batches
        mbar_arrive_expect_tx(&full_bar[0], kRecvBytes);
        mbar_arrive_expect_tx(&full_bar[1], kRecvBytes);
    }
    // shared::cluster address of every CTA's shared memory (offsets within a
    // CTA's window are linear, so buffers and barriers are base + offset)
    uint32_t r_base[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) r_base[r] = dsmem_map(smem_addr(smem), (uint32_t)r);
    constexpr uint32_t kFullOff = S::BAR_OFF + 3 * 8, kEmptyOff = S::BAR_OFF + 5 * 8;
    __syncthreads();
    cluster_sync_all();     // every barrier of the cluster is initialised before any remote use

    // Uses of the ring slots, receive buffers and their barriers are counted
    // over the whole kernel (u = kb + k), so they run on across the stream
    // segments of the cluster's share.
    auto give_up = [&]() {   // thread 0: record the error, stop all further work of this CTA
        atomicExch(args.err, 1);
        *sdead = 1;
    };
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
            carry[i] = (r >= 0 && r < n_raw) ? load_one_global<IN>(in, r * C + q * KS + tid) : make_float2(0.f, 0.f);
        }
        auto rows_of = [&](long long j) -> long long {
            const long long r = n_raw - (lo + j) * B;
            return r <= 0 ? 0 : (r < B ? r : B);
        };
        // raw batch j: the CTA's slice of rows [(lo+j)B, (lo+j)B + B), one bulk copy per row;
        // every use completes one phase of its slot's barrier (zero bytes past the stream)
        auto issue = [&](long long j) {
            const long long rows = rows_of(j);
            const long long u = kb + j;
            uint64_t* bar = &raw_bar[u & 1];
            mbar_expect_tx(bar, (uint32_t)(rows * KS * BIN));
            unsigned char* dst = ring + (u & 1) * S::SLOTB;
            const unsigned char* src = in + ((size_t)(lo + j) * B * C + (size_t)q * KS) * BIN;
            for (long long r = 0; r < rows; ++r)
                tma_load_1d(dst + r * KS * BIN, src + (size_t)r * C * BIN, KS * BIN, bar);
        };
        auto wait_raw = [&](long long j, uint64_t limit) -> bool {
            const long long u = kb + j;
            return mbar_wait_bounded(&raw_bar[u & 1], (uint32_t)((u >> 1) & 1), limit);
        };
        if (tid == 0 && !*sdead) {
            fence_proxy_async_smem();   // the slots were last read by an earlier segment's FIR
            issue(0);
            if (nraw_b > 1) issue(1);
        }

        for (long long k = 0; k <= nraw_b; ++k) {
            if (k < nraw_b) {
                const long long u = kb + k;
                // ------------------------------------------- wait for raw slot k
                if (tid == 0 && !*sdead) {
                    bool ok = wait_raw(k, kWaitLimitNs);
                    if (kb == 0 && k == 0 && q == 0 && (args.flags & FWD_INJECT_TIMEOUT))
                        ok = ok && mbar_wait_bounded(inj_bar, 0, kInjectedWaitNs);
                    if (!ok) {
                        for (long long j = k; j < k + 2 && j < nraw_b; ++j) wait_raw(j, kWaitLimitNs);
                        give_up();
                    }
                }
                __syncthreads();
                bool dead = *sdead != 0;
                // ----------------------------------------------------------- FIR
                unsigned long long acc[B];
#pragma unroll
                for (int j = 0; j < B; ++j) acc[j] = 0ull;
                if (!dead) {
                    const unsigned char* slot = ring + (u & 1) * S::SLOTB + tid * BIN;
                    float2 nxt[TM > 1 ? TM - 1 : 1];
#pragma unroll
                    for (int i = 0; i < B + TM - 1; ++i) {
                        const float2 x = (i < TM - 1) ? carry[i < TM - 1 ? i : 0]
                                                      : load_one_smem<IN>(slot + (size_t)(i - (TM - 1)) * KS * BIN);
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
                if (tid == 0 && !*sdead) {
                    if (k + 2 < nraw_b) {            // raw slot k is free: refill it
                        fence_proxy_async_smem();
                        issue(k + 2);
                    }
                    // receive buffers u&1 of every CTA are free once all receivers
                    // arrived on this CTA's empty barrier after use u-2
                    if (u >= 2 && !mbar_wait_cluster_bounded(&empty_bar[u & 1], (uint32_t)(((u >> 1) - 1) & 1),
                                                             kWaitLimitNs)) {
                        for (long long j = k + 1; j < k + 3 && j < nraw_b; ++j) wait_raw(j, kWaitLimitNs);
                        give_up();
                    }
                }
                __syncthreads();
                dead = *sdead != 0;
                // ------------------------------------ push: spectrum j -> CTA j / SPC
                if (!dead) {
                    const uint32_t boff = (uint32_t)((u & 1) * S::RBUF) + (uint32_t)(q * KS + tid) * 8;
#pragma unroll
                    for (int j = 0; j < B; ++j) {
                        const int r = j / SPC, sp = j % SPC;
                        st_async_f2(r_base[r] + boff + (uint32_t)(sp * C * 8), upk2(acc[j]),
                                    r_base[r] + kFullOff + (uint32_t)((u & 1) * 8));
                    }
                }
            }
            if (k >= 1) {
                // ---------------------------------------- DFT of batch k-1 (this CTA's spectra)
                const long long u = kb + k - 1;
                if (tid == 0 && !*sdead) {
                    if (!mbar_wait_cluster_bounded(&full_bar[u & 1], (uint32_t)((u >> 1) & 1), kWaitLimitNs)) {
                        for (long long j = k; j < k + 2 && j < nraw_b; ++j) wait_raw(j, kWaitLimitNs);
                        give_up();
                    }
                }
                __syncthreads();
                float2* buf = rbuf + (u & 1) * (SPC * C);
                const long long sbp = (lo + k - 1) * B - (T - 1) + q * SPC;   // output spectrum of buffer row 0
                const long long pvlo = *sdead ? vhi : vlo;                      // a CTA that gave up stores nothing
                static_for<NST>([&](auto p) {
                    fft_stage<C, SPC, NT, decltype(p)::value, OUT, true>(buf, tw_s, out, sbp, pvlo, vhi);
                });
                // the last stage synchronised the CTA after its reads: buffer u&1 is free
                if (tid == 0 && !*sdead) {
                    mbar_arrive_expect_tx(&full_bar[u & 1], kRecvBytes);   // it now expects use u+2
#pragma unroll
                    for (int r = 0; r < Q; ++r) mbar_arrive_remote(r_base[r] + kEmptyOff + (uint32_t)((u & 1) * 8));
                }
            }
        }
        kb += nraw_b;
    }
    __syncthreads();
    cluster_sync_all();   // no CTA leaves while a peer may still store to it or arrive on its barriers
}

}  // namespace ppf
