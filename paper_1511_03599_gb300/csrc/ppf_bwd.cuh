// ppf_bwd.cuh -- adjoint (backward pass) of the fused PFB for complex FP32
// input, in the conjugate-Wirtinger convention of PyTorch (for a real loss L
// and complex z, grad_z = dL/dRe z + i dL/dIm z).
//
// The forward map is Y = F y, y[s][c] = sum_t h[t][c] x[s+t][c] (Alg. 1,
// Eq. 2); it is complex-linear in x and real-linear in h, so with the
// incoming gradient G = grad_Y:
//   g_y = F^H G                          (unnormalised inverse DFT, sign +i)
//   grad_x[r][c] = sum_t h[t][c] g_y[r-t][c]            (transposed FIR)
//   grad_h[t][c] = sum_r Re(conj(g_y[r-t][c]) x[r][c])  (tap correlation)
// with g_y[s] = 0 outside 0 <= s < S.  Both sums run over raw rows r, so the
// work is partitioned by r: the batches of raw rows of all streams form one
// sequence (stream-major) and each CTA owns an equal contiguous share of it,
// which may span stream boundaries (every CTA of the grid busy whatever the
// stream count).  Within each stream segment of its share the CTA needs g_y
// rows back to r-(T-1) (carried in registers from the previous batch, or
// from one leading batch it inverse-transforms at the segment's start), and
// writes every grad_x row of the segment exactly once.  The tap gradient is
// accumulated per thread in registers, written as one partial per CTA, and
// summed over CTAs in a fixed order by a second kernel (deterministic: no
// floating-point atomics).
//
// Per CTA and batch of B raw rows: TMA copies of the G rows and the x rows
// of the batch into double-buffered shared-memory slots, the inverse DFT in
// place in the G slot (warp-local stages), then one thread per channel runs
// both sums over the batch rows.
#pragma once

#include "ppf_fwd.cuh"

#ifndef PPF_BWD_CARRY_SMEM
#define PPF_BWD_CARRY_SMEM 1
#endif

namespace ppf {

template <int C, int TM, int IN = IN_CF32>
struct BwdShape {
    static constexpr int NT = C;                                     // one channel per thread
    // C = 512 with 8/16-bit input and up to 8 taps: batches of 16 rows, so each
    // of the 16 warps owns a whole spectrum in the inverse DFT (no CTA
    // barriers between its stages); the per-channel sums run in two passes
    // of 8 rows to keep the carried state in registers
    static constexpr bool WIDE = C == 512 && IN != IN_CF32 && TM <= 8;
    static constexpr int B = WIDE ? 16 : 4096 / C;                   // raw rows per batch
    static constexpr int BF = WIDE ? 8 : B;                          // rows per pass of the channel sums
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr int SLOTB = B * C * 8;                          // complex FP32 rows of G of a batch
    static constexpr int XSLOTB = B * C * BIN;                       // raw rows of x of a batch
    static constexpr int NWARP = NT / 32;
    // spectra per warp in the inverse DFT; 0: the stages are spread over the
    // whole CTA (C = 512, where a batch has fewer spectra than warps)
    static constexpr int SPW = NWARP > 0 && B >= NWARP ? B / NWARP : 0;
    static constexpr int TWB = tw_size(C) * 8;                       // twiddle tables
    // WIDE with 8 taps: the 7 carried g_y rows wait in shared memory (one
    // column per thread) while the inverse DFT holds its 64 values per thread
    // in registers (+3 .. +4 %; with 4 taps the registers measured 3 % faster)
    static constexpr bool CARRY_SMEM = WIDE && TM >= 8 && PPF_BWD_CARRY_SMEM;
    static constexpr int CARRY_OFF = 2 * SLOTB + 2 * XSLOTB + TWB + 64;
    static constexpr int SMEM = CARRY_OFF + (CARRY_SMEM ? (TM - 1) * NT * 8 : 0);
    static constexpr bool FFT_OK = SPW > 0 ? (SPW * NWARP == B && (WIDE ? warp_fft_ok(C, SPW) : fft_items_fit(C, SPW, 32)))
                                           : C == 512;
    static constexpr bool OK = (C >= 64 && C <= 512) && (TM <= 16) && (BF >= TM - 1) && B % BF == 0 && FFT_OK;
};

struct BwdArgs {
    const float2* gY;        // incoming gradient, n_spectra*C per stream
    const void* x;           // forward input (the plan's input type), C*(n_spectra+T-1) samples per stream
    const float* taps;       // TM*C floats, tap-major, rows >= T zero
    const float2* tw;        // twiddle tables of the forward plan
    float2* gx;              // grad wrt x, same layout as x (nullptr: skip)
    float* partials;         // gridDim.x * TM * C tap-gradient partial sums
    int* err;
    long long n_spectra;
    long long gY_stride, x_stride;   // samples between streams
    long long n_streams;
    int T;
    int flags;
};

template <int C, int TM, int IN>
__global__ void __launch_bounds__(BwdShape<C, TM, IN>::NT, 1) pfb_bwd_kernel(BwdArgs args) {
    using S = BwdShape<C, TM, IN>;
    constexpr int NT = S::NT, B = S::B, BF = S::BF, NST = fft_stages(C), BIN = S::BIN;
    static_assert(S::OK, "shape not supported by the backward kernel");
    extern __shared__ __align__(128) unsigned char smem[];
    float2* gslot = reinterpret_cast<float2*>(smem);                    // [2][B][C] complex FP32
    unsigned char* xslot = smem + 2 * S::SLOTB;                         // [2][B][C] raw samples
    float2* tw_s = reinterpret_cast<float2*>(smem + 2 * S::SLOTB + 2 * S::XSLOTB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * S::SLOTB + 2 * S::XSLOTB + S::TWB);  // g0 g1 x0 x1 never
    volatile int* sflag = reinterpret_cast<volatile int*>(bars + 5);

    const int c = threadIdx.x;
    const long long n_spectra = args.n_spectra;
    const int T = args.T;
    const long long n_raw = n_spectra + T - 1;
    const long long nbt = (n_raw + B - 1) / B;        // batches of raw rows per stream
    const long long U = nbt * args.n_streams;          // batches of all streams
    const long long u0 = (long long)blockIdx.x * U / gridDim.x;
    const long long u1 = (long long)(blockIdx.x + 1) * U / gridDim.x;

    // tap-gradient accumulators (over all segments); the taps of channel c are
    // loaded (from L1) as (h, h) pairs before each batch's channel sums, so
    // they are not live across the inverse DFT
    unsigned long long acch[TM];
#pragma unroll
    for (int t = 0; t < TM; ++t) acch[t] = 0ull;
    for (int i = c; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
    if (c == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        *sflag = 0;
    }
    __syncthreads();

    // Uses of the G slots and of the x slots in earlier segments: slot use n
    // (counted over the whole kernel) waits for phase n of its barrier.
    long long gbase = 0, xbase = 0;
    for (long long u = u0; u < u1;) {
        const long long strm = u / nbt;
        const long long lo = u - strm * nbt;
        const long long hi = (u1 - strm * nbt < nbt) ? u1 - strm * nbt : nbt;
        u = strm * nbt + hi;
        const long long nb = hi - lo;
        const float2* gY = args.gY + (size_t)strm * args.gY_stride;
        const unsigned char* x = static_cast<const unsigned char*>(args.x) + (size_t)strm * args.x_stride * BIN;
        float2* gx = args.gx ? args.gx + (size_t)strm * args.x_stride : nullptr;

        unsigned long long carry[TM > 1 ? TM - 1 : 1];     // g_y rows (first row) - (TM-1) .. -1
        constexpr bool CSMEM = S::CARRY_SMEM;
        unsigned long long* scarry = reinterpret_cast<unsigned long long*>(smem + S::CARRY_OFF) + c;   // [i * NT]
#pragma unroll
        for (int i = 0; i < TM - 1; ++i) {
            if constexpr (CSMEM) scarry[i * NT] = 0ull;
            else carry[i] = 0ull;
        }

        // iterations: k = k0 (a leading batch that only fills the carry) .. nb-1
        const long long k0 = (lo > 0 && TM > 1) ? -1 : 0;
        const long long nit = nb - k0;
        auto g_rows = [&](long long j) -> long long {     // valid G rows of absolute batch j
            const long long r = n_spectra - j * B;
            return r <= 0 ? 0 : (r < B ? r : B);
        };
        auto x_rows = [&](long long j) -> long long {
            const long long r = n_raw - j * B;
            return r <= 0 ? 0 : (r < B ? r : B);
        };
        // G slots are indexed by the iteration it; x slots by the x batch k
        // (there is no x batch in the leading iteration).  Every use of a
        // slot completes one phase of its barrier, also a use with nothing to
        // copy (the last batch of a stream may hold no G row): the arrival
        // then expects zero bytes, so uses and phases stay in step across
        // the segments of the CTA's share.
        auto issue = [&](long long it) {                   // iteration it = k - k0
            const long long k = it + k0, j = lo + k;
            const int q = (int)((gbase + it) & 1);
            const long long gr = g_rows(j);
            mbar_expect_tx(&bars[q], (uint32_t)(gr * C * 8));
            if (gr > 0) tma_load_1d(gslot + q * B * C, gY + (size_t)j * B * C, (uint32_t)(gr * C * 8), &bars[q]);
            if (k >= 0) {
                const long long xr = x_rows(j);
                const int qx = (int)((xbase + k) & 1);
                mbar_expect_tx(&bars[2 + qx], (uint32_t)(xr * C * BIN));
                if (xr > 0)
                    tma_load_1d(xslot + qx * S::XSLOTB, x + (size_t)j * B * C * BIN, (uint32_t)(xr * C * BIN),
                                &bars[2 + qx]);
            }
        };
        auto wait_it = [&](long long it, uint64_t limit) -> bool {
            const long long k = it + k0;
            const long long gn = gbase + it, xn = xbase + k;
            bool ok = mbar_wait_bounded(&bars[gn & 1], (uint32_t)((gn >> 1) & 1), limit);
            if (k >= 0) ok = mbar_wait_bounded(&bars[2 + (xn & 1)], (uint32_t)((xn >> 1) & 1), limit) && ok;
            return ok;
        };
        if (c == 0) {
            fence_proxy_async_smem();   // slots written by an earlier segment's inverse DFT
            issue(0);
            if (nit > 1) issue(1);
        }

        for (long long it = 0; it < nit; ++it) {
            const long long k = it + k0, j = lo + k;
            float2* gs = gslot + ((gbase + it) & 1) * B * C;
            const unsigned char* xs = xslot + ((xbase + k) & 1) * S::XSLOTB;
            if (c == 0) {
                bool ok = wait_it(it, kWaitLimitNs);
                if (gbase == 0 && it == 0 && (args.flags & FWD_INJECT_TIMEOUT))
                    ok = ok && mbar_wait_bounded(&bars[4], 0, kInjectedWaitNs);
                if (!ok) {
                    for (long long i2 = it; i2 < it + 2 && i2 < nit; ++i2) wait_it(i2, kWaitLimitNs);
                    atomicExch(args.err, 1);
                    *sflag = 1;
                }
            }
            __syncthreads();
            if (*sflag) return;
            // g_y = F^H G for the B rows of the batch, in place (warp-local stages)
            static_for<NST>([&](auto p) {
                fft_stage<C, B, NT, decltype(p)::value, OUT_CF32, true, S::SPW, true>(gs, tw_s, nullptr, 0, 0, 0);
            });
            __syncthreads();
            unsigned long long hh[TM];
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                const float h = __ldg(args.taps + t * C + c);
                hh[t] = pk2(h, h);
            }
            // one thread per channel, in passes of BF rows: sequence g_i = carried rows
            // (i < TM-1) then the pass's rows
            for (int hf = 0; hf < B / BF; ++hf) {
            const long long row0 = j * B + hf * BF;       // first raw row (and G row) of the pass
            unsigned long long gxa[BF];
#pragma unroll
            for (int r = 0; r < BF; ++r) gxa[r] = 0ull;
            unsigned long long gseq[BF + TM - 1];
#pragma unroll
            for (int i = 0; i < TM - 1; ++i) gseq[i] = CSMEM ? scarry[i * NT] : carry[i];
            const float2* gsc = gs + (size_t)hf * BF * C + c;
            const unsigned char* xsc = xs + ((size_t)hf * BF * C + c) * BIN;
            if (row0 + BF <= n_spectra && T == TM) {        // whole batch, every tap: no checks
#pragma unroll
                for (int r = 0; r < BF; ++r) {
                    const float2 g = gsc[r * C];
                    gseq[TM - 1 + r] = pk2(g.x, g.y);
                }
                if (k >= 0) {
#pragma unroll
                    for (int r = 0; r < BF; ++r) {
                        const float2 xv = load_one_smem<IN>(xsc + (size_t)r * C * BIN);
                        const unsigned long long xp = pk2(xv.x, xv.y);
#pragma unroll
                        for (int t = 0; t < TM; ++t) {
                            const unsigned long long g = gseq[TM - 1 + r - t];
                            ffma2(gxa[r], hh[t], g);
                            ffma2(acch[t], g, xp);
                        }
                    }
                    if (gx != nullptr) {
                        float2* gxr = gx + (size_t)row0 * C + c;
#pragma unroll
                        for (int r = 0; r < BF; ++r) gxr[r * C] = upk2(gxa[r]);
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < BF; ++r) {
                    const float2 g = (row0 + r < n_spectra) ? gsc[r * C] : make_float2(0.f, 0.f);
                    gseq[TM - 1 + r] = pk2(g.x, g.y);
                }
                if (k >= 0) {
#pragma unroll
                    for (int r = 0; r < BF; ++r) {
                        const float2 xv = (row0 + r < n_raw) ? load_one_smem<IN>(xsc + (size_t)r * C * BIN)
                                                             : make_float2(0.f, 0.f);
                        const unsigned long long xp = pk2(xv.x, xv.y);
#pragma unroll
                        for (int t = 0; t < TM; ++t) {
                            if (t < T) {
                                const unsigned long long g = gseq[TM - 1 + r - t];
                                ffma2(gxa[r], hh[t], g);        // grad_x[r] += h[t] g_y[r-t]
                                ffma2(acch[t], g, xp);          // (g.re x.re, g.im x.im)
                            }
                        }
                    }
                    if (gx != nullptr) {
                        float2* gxr = gx + (size_t)row0 * C + c;
#pragma unroll
                        for (int r = 0; r < BF; ++r)
                            if (row0 + r < n_raw) gxr[r * C] = upk2(gxa[r]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < TM - 1; ++i) {
                if constexpr (CSMEM) scarry[i * NT] = gseq[BF + i];
                else carry[i] = gseq[BF + i];
            }
            }
            __syncthreads();
            if (c == 0 && it + 2 < nit) {
                fence_proxy_async_smem();
                issue(it + 2);
            }
        }
        gbase += nit;
        xbase += nb;
    }
    float* part = args.partials + (size_t)blockIdx.x * TM * C;
#pragma unroll
    for (int t = 0; t < TM; ++t) {
        const float2 a = upk2(acch[t]);
        part[t * C + c] = a.x + a.y;
    }
}

// grad_h[t*C + c] = sum over CTAs, in CTA order, of the partial sums.  When
// the status word is set (a bounded wait of the adjoint gave up, so some
// partial rows were never written), every element is NaN instead.
static __global__ void pfb_bwd_reduce_kernel(const float* __restrict__ partials, int nparts, int TC, int TMC,
                                      const int* __restrict__ err, float* __restrict__ grad_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TC) return;
    if (*err != 0) {
        grad_h[i] = __int_as_float(0x7fc00000);
        return;
    }
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += partials[(size_t)p * TMC + i];
    grad_h[i] = s;
}

struct BwdInfo {
    int threads, batch, smem;
    const void* fn;
};

template <int C, int TM, int IN>
inline BwdInfo bwd_info() {
    using S = BwdShape<C, TM, IN>;
    if constexpr (S::OK) return BwdInfo{S::NT, S::B, S::SMEM, reinterpret_cast<const void*>(&pfb_bwd_kernel<C, TM, IN>)};
    else return BwdInfo{0, 0, 0, nullptr};
}

template <int C, int TM, int IN>
inline cudaError_t bwd_launch(const BwdArgs& a, int grid, cudaStream_t st) {
    using S = BwdShape<C, TM, IN>;
    if constexpr (S::OK) {
        pfb_bwd_kernel<C, TM, IN><<<grid, S::NT, S::SMEM, st>>>(a);
        return cudaPeekAtLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

}  // namespace ppf
