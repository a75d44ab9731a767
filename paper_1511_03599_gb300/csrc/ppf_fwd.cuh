// ppf_fwd.cuh -- the fused polyphase filter bank forward kernel.
//
// One persistent CTA loops over batches of B consecutive output spectra.
// Per batch:
//   1. FIR (Alg. 1): each thread owns a channel pair and a segment of L
//      output spectra; it reads the L+T-1 raw samples of its pair from the
//      TMA ring of raw batches in shared memory (where the ring fits beside
//      the batch; else straight from global memory, warmed in L2 ahead) --
//      each raw sample is converted to FP32 once per segment and reused by
//      all T taps in registers, the T-1 rows shared with the previous
//      segment (the halo of Sec. 3.2) are read again -- and writes the
//      filtered spectra y to shared memory.  y never goes to global memory.
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
// C = 2^k: two stages up to 1024, three above.  C = 3 * 2^k: a radix-3
// stage first, then two power-of-two stages.
constexpr bool is_c3(int C) { return C == 384 || C == 768 || C == 1536 || C == 3072; }
constexpr int fft_stages(int C) { return (C >= 2048 || is_c3(C)) ? 3 : 2; }
constexpr int fft_radix(int C, int p) {
    switch (C) {
        case 384:  return p == 0 ? 3 : p == 1 ? 8 : 16;
        case 768:  return p == 0 ? 3 : 16;
        case 1536: return p == 0 ? 3 : p == 1 ? 32 : 16;
        case 3072: return p == 0 ? 3 : 32;
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
// Physical index inside one spectrum slot of buffer A_p.  Buffers read by
// a non-final stage are plain; the buffer read by the last stage (rows of
// R = R_last elements, read column-wise by lanes walking consecutive rows
// and written row-wise) is XOR-swizzled within each row so both access
// patterns hit 16 distinct 8-byte bank pairs per half-warp.
//
// LAYOUT 1 pads the rows of that last buffer instead (row stride R + 1, an
// odd number of elements, also conflict-free for both patterns): every
// access is then a per-lane base plus a compile-time offset, with no XOR per
// access.  It needs a spectrum span of C + C/R elements (spec_span); the
// carry kernel picks the layout per shape.
constexpr int last_radix(int C) { return fft_radix(C, fft_stages(C) - 1); }
template <int C, int LAYOUT>
constexpr int spec_span() { return LAYOUT == 1 ? C + C / last_radix(C) : C; }

template <int C, int P, int LAYOUT = 0>
__device__ __forceinline__ int phys(int i) {
    constexpr int NST = fft_stages(C);
    if constexpr (P > 0 && P == NST - 1 && LAYOUT == 2) {
        // 16-byte chunks (element pairs) of each row of R >= 16 elements
        // XOR-swizzled with the row index mod 8: a lane reading a whole row
        // as 16-byte loads and lanes walking 8 consecutive rows hit 8
        // distinct chunks of the 128-byte bank window, and a row written
        // element by element stays one contiguous row
        constexpr int R = fft_radix(C, P);
        static_assert(R >= 16, "pair-chunk swizzle needs rows of at least 16 elements");
        const int row = i / R, col = i % R;
        return row * R + (((col >> 1) ^ (row & 7)) << 1) + (col & 1);
    } else if constexpr (P > 0 && P == NST - 1 && LAYOUT == 1) {
        constexpr int R = fft_radix(C, P);
        return (i / R) * (R + 1) + i % R;
    } else if constexpr (P > 0 && P == NST - 1) {
        constexpr int R = fft_radix(C, P);
        constexpr int RPG = R >= 16 ? 1 : 16 / R;   // rows sharing one 16-element bank group
        return i ^ (((i / R) / RPG) & (R - 1));
    } else if constexpr (P > 0) {
        // A middle stage reads, per prefix row of N_P elements, R groups of
        // NN = N_{P+1} consecutive elements.  With NN < 16 one half-warp spans
        // G = 16/NN rows whose groups fall on the same banks; XOR the group
        // index with the row index mod G so they fall on different ones.
        constexpr int NP = fft_n(C, P), R = fft_radix(C, P), NN = NP / R;
        if constexpr (NN < 16 && 16 / NN <= R && (NN & (NN - 1)) == 0 && (R & (R - 1)) == 0) {
            constexpr int G = 16 / NN;
            return i ^ (((i / NP) % G) * NN);
        } else {
            return i;
        }
    } else {
        return i;
    }
}
// Twiddle tables: stage p (p < P-1) holds W_{N_p}^{b k}, k = 1 .. R_p-1, for
// the N_{p+1} columns b: (R_p - 1) * N_{p+1} entries at [(k-1)*N_{p+1} + b],
// so lanes with consecutive b read consecutive entries.  (A layout with the
// entries of one column adjacent, read as 16-byte (k, k+1) pairs, measured
// slower at C = 512.)
constexpr int tw_offset(int C, int p) {
    int off = 0;
    for (int q = 0; q < p; ++q) off += (fft_n(C, q) / fft_radix(C, q)) * (fft_radix(C, q) - 1);
    return off;
}
constexpr int tw_size(int C) { return tw_offset(C, fft_stages(C) - 1); }

// v[k] *= W_{N_p}^{b k} for k = 1 .. R-1; tw_stage is stage p's table (NN = N_{p+1} columns)
template <int R, int NN, bool TW_SMEM>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[R], const float2* __restrict__ tw_stage, int b) {
#pragma unroll
    for (int k = 1; k < R; ++k) {
        const float2* p = tw_stage + (k - 1) * NN + b;
        v[k] = cmul(v[k], TW_SMEM ? *p : __ldg(p));
    }
}

// ------------------------------------------------------------ launch shape
// Raw batches are copied with an L2 evict-first policy (each is read once):
// +0.1-0.3 % on every measured carry-kernel shape; the output's lines stay
// in L2 longer.
#ifndef PPF_TMA_EVICT_FIRST
#define PPF_TMA_EVICT_FIRST 1
#endif
#ifndef PPF_PINGPONG
#define PPF_PINGPONG 1
#endif
#ifndef PPF_PINGPONG_256
#define PPF_PINGPONG_256 1       // also for 256 threads at C = 1536 (fp32 +43 %; C = 768 lost 1.5 %)
#endif
#ifndef PPF_PACKED_MIN_L
#define PPF_PACKED_MIN_L 4       // shortest FIR segment that takes the packed channel-pair path
#endif
#ifndef PPF_WIDE_1024
#define PPF_WIDE_1024 1          // 512 threads (one CTA per SM) for fp32 input at C = 1024, T = 9..16
#endif
#ifndef PPF_RING_TIGHT
#define PPF_RING_TIGHT 1         // a ring of HS + 1 slots where only that fits beside the batch
#endif
#ifndef PPF_GENERIC_B2048
#define PPF_GENERIC_B2048 0      // spectra per batch of the generic kernel at C = 2048 (0: chosen below)
#endif
#ifndef PPF_GENERIC_B1024_SHORT
#define PPF_GENERIC_B1024_SHORT 4   // spectra per batch at C = 1024, 16/32-bit input, up to 4 taps
#endif
#ifndef PPF_GENERIC_B3072
#define PPF_GENERIC_B3072 4      // spectra per batch of the generic kernel at C = 3072
#endif
#ifndef PPF_GENERIC_B4096
#define PPF_GENERIC_B4096 0      // spectra per batch of the generic kernel at C = 4096 (0: chosen below)
#endif
// Largest dynamic shared memory of one generic-kernel CTA (two CTAs per SM
// with 256 threads, one with 512).
constexpr int generic_smem_cap(int NT) { return (NT == 256 ? 113 * 1024 : 226 * 1024) - 128; }
// Whether the direct-load mode can run its DFT stages out of place between
// two spectra buffers (512 threads, or 256 from C = 1536).
constexpr bool generic_pingpong_ok(int C, int B, int NT) {
    return PPF_PINGPONG && (NT == 512 || (PPF_PINGPONG_256 && C >= 1536)) && 2 * B * C * 8 <= generic_smem_cap(NT);
}
// Whether a ring without the refill slot is allowed: where the halo spans two
// or more batches, or where the alternative is plain direct loads (no
// out-of-place mode).  A 2-slot ring lost to the out-of-place mode (C = 3072
// int16 T = 4: 160 vs 170 GS/s) but beat plain direct loads (C = 1024 fp32
// T = 4: 218 vs 175).
constexpr bool generic_ring_tight_ok(int C, int TM, int B, int NT) {
    return PPF_RING_TIGHT && (TM - 1 > B || !generic_pingpong_ok(C, B, NT));
}
// Whether the generic kernel's TMA ring fits one CTA's shared memory beside a
// B-spectrum batch of filtered values: HS = ceil((T-1)/B) halo slots (1 when
// T-1 <= B) plus the slot being read and, where room is left, one of slack
// for the refill (`slack` = 1), else none (0).  The ring also needs the FIR
// segment to cover the whole batch when the halo spans several batches
// (segments of min(B, 16) outputs at these channel counts, T <= 16).
constexpr bool generic_ring_fits(int C, int TM, int bin, int B, int NT, int slack) {
    const int hs = TM - 1 <= B ? 1 : (TM - 1 + B - 1) / B;
    const bool one_segment = B <= 16 && TM <= 16;
    return (TM - 1 <= B || one_segment) && B * C * 8 + (hs + 1 + slack) * B * C * bin + 64 <= generic_smem_cap(NT);
}
constexpr bool generic_ring_fits_any(int C, int TM, int bin, int B, int NT) {
    return generic_ring_fits(C, TM, bin, B, NT, 1) ||
           (generic_ring_tight_ok(C, TM, B, NT) && generic_ring_fits(C, TM, bin, B, NT, 0));
}
// Spectra per batch of the generic kernel at C = 2048 and 4096: the larger
// batch where its ring fits (fewer halo rows re-read and fewer barriers per
// spectrum: C = 2048 int8 T = 8, 8 spectra: 265 GS/s vs 213 with 4;
// C = 4096 int8 T = 8, 4 spectra: 235 vs 184 with 2), else the smaller one
// where that keeps the ring (C = 4096 int8 T = 16: 128 GS/s with a 10-slot
// ring of 2-spectrum batches vs 113 without a ring at 4), else the larger
// (C = 4096 int16 T = 16, direct loads: 105 vs 62).  Beyond 16 taps (no
// ring at these sizes) the smaller batch, with its out-of-place DFT stages.
constexpr int generic_batch_large(int C, int TM, int bin, int NT) {
    const int big = C >= 4096 ? 4 : 8;
    return TM > 16 ? big / 2
         : generic_ring_fits_any(C, TM, bin, big, NT) ? big
         : generic_ring_fits_any(C, TM, bin, big / 2, NT) ? big / 2
         : big * C * 8 <= generic_smem_cap(NT) ? big : big / 2;
}

template <int C, int TM, int IN, int NTO = 0>
struct FwdShape {
    // threads per CTA: 512 from C = 2048, and for fp32 input at C = 1024 with
    // 9-16 taps (out-of-place DFT stages: 149 vs 123 GS/s at T = 16)
    // (two CTAs of 256 threads per SM at C = 2048/3072, on half the batch,
    // measured slower: 256 vs 265 GS/s at C = 2048 int8 T = 8, 133 vs 152 at 3072)
    static constexpr int NT = NTO ? NTO : (C >= 2048 || (C == 1024 && IN == IN_CF32 && TM == 16 && PPF_WIDE_1024)) ? 512 : 256;
    static constexpr int PAIRS = C / 2;
    // spectra per batch: 64 KB of filtered spectra (48 KB for C = 3 * 2^k),
    // 64-128 KB at C = 2048 and 4096 (generic_batch_large); half that where
    // it lets the TMA ring fit beside the batch: 16/32-bit input at C = 32
    // (fp32 T = 8: 244 vs 120 GS/s; int16 T = 8: 233 vs 148) and 16-tap
    // int16 input at C = 768 (140 vs 102)
    static constexpr int B = (C == 4096) ? (PPF_GENERIC_B4096 ? PPF_GENERIC_B4096 : generic_batch_large(C, TM, InTraits<IN>::bytes, NT))
                           : (C == 2048) ? (PPF_GENERIC_B2048 ? PPF_GENERIC_B2048 : generic_batch_large(C, TM, InTraits<IN>::bytes, NT))
                           : C == 3072 ? PPF_GENERIC_B3072
                           : (C == 1024 && IN != IN_CI8 && TM <= 4) ? PPF_GENERIC_B1024_SHORT
                           : (C == 32 && IN != IN_CI8) ? 128
                           : (C == 768 && IN == IN_CI16 && TM == 16) ? 4
                           : is_c3(C) ? 16 * 384 / C : 8192 / C;
    // large-T FIR order (see fir_segment): tap chunks for narrow input at C <= 512
    static constexpr bool CHUNK = TM > 16 && IN != IN_CF32 && C <= 512;
    static constexpr int L0 = (TM >= 32 && !CHUNK) || (C == 32 && IN != IN_CI8) ? 8 : 16;
    static constexpr int L = L0 < B ? L0 : B;                        // FIR segment (outputs)
    static constexpr int G = B / L;                                  // segments per batch
    static constexpr int FIR_ITEMS = PAIRS * G;                      // (pair, segment) items
    static constexpr int FPT = (FIR_ITEMS + NT - 1) / NT;           // FIR items per thread
    static constexpr bool FIR_EXACT = FIR_ITEMS % NT == 0;
    static constexpr int YBYTES = B * C * 8;                         // filtered spectra of a batch
    static constexpr int TWBYTES = tw_size(C) * 8;
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr int SLOTB = B * C * BIN;                        // raw bytes of one batch
    static constexpr int CTA_SMEM_MAX = generic_smem_cap(NT);
    // TMA ring: every raw batch is copied into shared memory once; the FIR of
    // batch k reads slot k and the T-1 halo rows from the HS slots after it
    // (HS = 1 when T-1 <= B; a deeper ring where the halo spans several
    // batches -- large C, where B is small -- and one segment covers the batch).
    static constexpr int HS = TM - 1 <= B ? 1 : (TM - 1 + B - 1) / B;    // halo slots
    // ring slots: HS + 2 (one batch of slack for the refill), or HS + 1 where
    // only that fits, or where only that leaves room for the twiddle table
    // (the refill of the slot freed by batch k's FIR then has batch k's DFT
    // stages to land before batch k+1's FIR reads it; twiddles in shared
    // memory beside a 2-slot ring measured +2 .. +3 % at C = 2048 and 4096)
    static constexpr bool NS_TIGHT_FITS = YBYTES + (HS + 1) * SLOTB + 64 <= CTA_SMEM_MAX;
    static constexpr bool NS_TIGHT_FOR_TW = YBYTES + (HS + 2) * SLOTB + 64 + TWBYTES > CTA_SMEM_MAX &&
                                            YBYTES + (HS + 1) * SLOTB + 64 + TWBYTES <= CTA_SMEM_MAX;
    static constexpr int NS = (generic_ring_tight_ok(C, TM, B, NT) && NS_TIGHT_FITS &&
                               (YBYTES + (HS + 2) * SLOTB + 64 > CTA_SMEM_MAX || NS_TIGHT_FOR_TW)) ? HS + 1 : HS + 2;
    static constexpr bool RING = (TM - 1 <= B || (G == 1 && TM <= 16)) && (YBYTES + NS * SLOTB + 64 <= CTA_SMEM_MAX);
    // direct-load mode with 512 threads (and at C = 1536 with 256): two
    // filtered-spectra buffers, so the DFT stages run out of place (read one
    // buffer, write the other), one CTA barrier per stage instead of two
    // (fp32 at C = 3072: 93 -> 131 GS/s, at C = 1536: 94 -> 135); with the
    // ring the second buffer would push the twiddles out of shared memory,
    // which measured 1 % slower at C = 4096
    static constexpr bool PINGPONG = generic_pingpong_ok(C, B, NT) && !RING;
    static constexpr int YB = PINGPONG ? 2 * YBYTES : YBYTES;        // bytes of the spectra buffers
    static constexpr bool TW_SMEM = YB + (RING ? NS * SLOTB + 64 : 0) + TWBYTES <= CTA_SMEM_MAX;
    static constexpr int RING_OFF = YB + (TW_SMEM ? TWBYTES : 0);
    static constexpr int SMEM = RING_OFF + (RING ? NS * SLOTB + 64 : 0);
    // each thread keeps one channel pair for the whole run: taps stay in registers
    static constexpr bool TAPS_IN_REGS = (FPT == 1) && (TM <= 16) && (NT % PAIRS == 0);
    static_assert(FPT >= 1 && (FIR_EXACT || is_c3(C)), "FIR items must divide evenly");
    static_assert(SLOTB % 16 == 0 && YBYTES % 16 == 0 && TWBYTES % 16 == 0, "16-byte alignment");
    static_assert(SMEM <= CTA_SMEM_MAX, "the batch and its ring must fit one CTA's shared memory");
};

enum FwdFlags { FWD_INJECT_TIMEOUT = 1 };
constexpr uint64_t kWaitLimitNs = 2000000000ull;     // 2 s
constexpr uint64_t kInjectedWaitNs = 2000000ull;     // 2 ms

struct FwdArgs {
    const void* in;          // raw streams, C*(n_spectra+T-1) samples each
    void* out;               // n_spectra*C outputs per stream
    long long in_stride;     // samples between consecutive input streams
    long long out_stride;    // samples between consecutive output streams
    long long n_streams;     // streams; the carry kernel splits the grid evenly over them (the grid is a
                             // multiple of n_streams), the others share the batches of all streams
                             // equally among their work units (CTAs, or clusters)
    const float* taps;       // TM*C floats, tap-major, rows >= T are zero
    const float2* tw;        // twiddle tables, tw_size(C) entries
    int* err;                // device status word: 1 = a bounded wait gave up
    long long n_spectra;
    int T;
    int flags;               // FwdFlags (testing aid)
};

// Thread-group policies: which threads run a body and how they synchronise.
// CtaGroup: the whole CTA (__syncthreads).  HalfGroup<N>: threads
// [g*N, g*N + N) form group g and synchronise on named barrier g + 1, so the
// groups of one CTA run independent bodies (the multi-beam kernel).
struct CtaGroup {
    __device__ static __forceinline__ int tid() { return threadIdx.x; }
    __device__ static __forceinline__ void sync() { __syncthreads(); }
};
template <int N>
struct HalfGroup {
    __device__ static __forceinline__ int tid() { return threadIdx.x % N; }
    __device__ static __forceinline__ void sync() {
        asm volatile("bar.sync %0, %1;" ::"r"((int)(threadIdx.x / N) + 1), "n"(N) : "memory");
    }
};

// One FFT stage over the whole batch held in shared memory.
// Output spectrum of batch row sp is sb + sp; it is stored when it lies in [vlo, vhi).
// SPW > 0: warp-local mode, warp w owns batch rows [w*SPW, (w+1)*SPW) in every
// stage, so the stages synchronise with __syncwarp only; SPW == 0: the items
// of a stage are spread over the whole CTA and __syncthreads separates them.
// INV: the unnormalised inverse DFT (sign +i) computed as conj(DFT(conj(.)));
// its last stage writes the result back into the spectrum's own row of
// ybuf in natural order instead of to global memory.
template <int C, int B, int NT, int P, int OUT, bool TW_SMEM, int SPW = 0, bool INV = false, bool SMEM_OUT = false,
          int LAYOUT = 0, class GRP = CtaGroup, bool OOP = false>
__device__ __forceinline__ void fft_stage(float2* __restrict__ ybuf, const float2* __restrict__ tws,
                                          void* __restrict__ out, long long sb, long long vlo, long long vhi,
                                          float2* __restrict__ dbuf = nullptr) {
    constexpr int NST = fft_stages(C);
    constexpr int R = fft_radix(C, P);
    constexpr int NP = fft_n(C, P);
    constexpr int NN = NP / R;                 // N_{p+1}
    constexpr int PP = C / NP;                 // prefixes at this stage
    constexpr int ITEMS = C / R;               // items per spectrum
    constexpr int WORKERS = SPW > 0 ? 32 : NT;
    constexpr int TOTAL = (SPW > 0 ? SPW : B) * ITEMS;
    constexpr int IPT = (TOTAL + WORKERS - 1) / WORKERS;        // items per thread
    constexpr bool EXACT = IPT * WORKERS == TOTAL;
    constexpr int SPAN = spec_span<C, LAYOUT>();   // elements per spectrum in ybuf
    static_assert(!(LAYOUT >= 1 && (INV || SMEM_OUT)), "padded or pair-swizzled rows only for the forward stores to HBM");
    static_assert(!(OOP && (INV || SMEM_OUT || SPW > 0)), "out-of-place stages only for the CTA-wide forward");
    static_assert(EXACT || (SPW == 0 && is_c3(C)) || TOTAL < WORKERS,
                  "items must divide evenly (a warp or CTA may leave threads idle)");
    const int gtid = GRP::tid();
    const int wid = SPW > 0 ? (gtid & 31) : gtid;
    const int sp0 = SPW > 0 ? (gtid >> 5) * SPW : 0;
    auto sync = [] {
        if constexpr (SPW > 0) __syncwarp();
        else GRP::sync();
    };

    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = wid + it * WORKERS;
        if (!EXACT && item >= TOTAL) break;
        const int sp = sp0 + item / ITEMS, e = item % ITEMS;
        const int b = e % NN, prefix = e / NN;
        const float2* src = ybuf + sp * SPAN;
        if constexpr (LAYOUT == 2 && P == NST - 1 && NN == 1) {
            // the item's whole row, as 16-byte element pairs
#pragma unroll
            for (int a = 0; a < R; a += 2) {
                const float4 q = *reinterpret_cast<const float4*>(src + phys<C, P, LAYOUT>(prefix * NP + a));
                v[it][a] = make_float2(q.x, q.y);
                v[it][a + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int a = 0; a < R; ++a) {
                v[it][a] = src[phys<C, P, LAYOUT>(prefix * NP + NN * a + b)];
                if constexpr (INV && P == 0) v[it][a].y = -v[it][a].y;
            }
        }
    }
    // every read of this stage is done before anything is overwritten; OOP
    // (out of place): a non-last stage writes to dbuf, a last stage stores to
    // global memory, and the caller orders the buffer's next writer after
    // these reads with a barrier of its own
    if constexpr (!OOP) sync();
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int item = wid + it * WORKERS;
        if (!EXACT && item >= TOTAL) break;
        const int sp = sp0 + item / ITEMS, e = item % ITEMS;
        const int b = e % NN, prefix = e / NN;
        dft_reg<R>(v[it]);
        if constexpr (P + 1 < NST) {
            apply_twiddles<R, NN, TW_SMEM>(v[it], tws + tw_offset(C, P), b);
            float2* dst = (OOP ? dbuf : ybuf) + sp * SPAN;
#pragma unroll
            for (int k = 0; k < R; ++k) dst[phys<C, P + 1, LAYOUT>((prefix + PP * k) * NN + b)] = v[it][k];
        } else if constexpr (INV) {
            float2* dst = ybuf + sp * C;
#pragma unroll
            for (int k = 0; k < R; ++k) dst[prefix + PP * k] = make_float2(v[it][k].x, -v[it][k].y);
        } else if constexpr (SMEM_OUT) {   // natural order, output type, row stride C elements
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if constexpr (OUT == OUT_CF32) {
                    ybuf[sp * C + prefix + PP * k] = v[it][k];
                } else {
                    reinterpret_cast<__half2*>(ybuf)[sp * C + prefix + PP * k] = __float22half2_rn(v[it][k]);
                }
            }
        } else {
            const long long s = sb + sp;
            if (s >= vlo && s < vhi) {
#pragma unroll
                for (int k = 0; k < R; ++k) store_out<OUT>(out, s * C + prefix + PP * k, v[it][k]);
            }
        }
    }
    if constexpr (P + 1 < NST || INV) sync();
}

// Where the FIR reads raw samples of channel pair cp from: rows are relative
// to the first raw spectrum of the batch (row r feeds outputs r-T+1 .. r).
template <int C, int IN, bool RING, int B, int HS = 1>
struct RawSrc {
    static constexpr int BIN = InTraits<IN>::bytes;
    static constexpr bool kRing = RING;
    // ring: shared-memory slots of the batch and of the HS batches after it
    const unsigned char* sl[HS + 1];
    // direct: global stream
    const void* in;
    long long row0, n_raw;
    int cp;

    __device__ __forceinline__ float4 load(int r) const {
        if constexpr (RING) {
            if constexpr (HS == 1) {
                const unsigned char* p = (r < B) ? sl[0] + (size_t)r * C * BIN : sl[1] + (size_t)(r - B) * C * BIN;
                return load_pair_smem<IN>(p);
            } else {
                return load_pair_smem<IN>(sl[r / B] + (size_t)(r % B) * C * BIN);   // r is a compile-time row here
            }
        } else {
            const long long rr = row0 + r;
            return (rr < n_raw) ? load_pair_global<IN>(in, rr * C + 2 * cp) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // rows [r0, r0 + n) all inside the stream: load_inside needs no check
    __device__ __forceinline__ bool inside(int r0, int n) const {
        if constexpr (RING) return true;
        else return row0 + r0 + n <= n_raw;
    }
    __device__ __forceinline__ float4 load_inside(int r) const {
        if constexpr (RING) return load(r);
        else return load_pair_global<IN>(in, (row0 + r) * C + 2 * cp);
    }
};

__device__ __forceinline__ void fma_pair(float4& acc, float2 h, float4 x) {
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.y = fmaf(h.x, x.y, acc.y);
    acc.z = fmaf(h.y, x.z, acc.z);
    acc.w = fmaf(h.y, x.w, acc.w);
}

// FIR (Alg. 1) of channel pair cp for the L output spectra whose first raw
// row is r0 (relative to the batch):
//   acc[j] = sum_{t<T} h[t][cp] * x[r0 + j + t][cp]
// Every raw sample of the segment (L+T-1 of them) is loaded and converted
// once; the taps are applied in ascending t for every output.
template <int TM, int IN, int L, int PAIRS, bool TAPS_IN_REGS, bool CHUNK, class Src>
__device__ __forceinline__ void fir_segment(const Src& src, const float2* __restrict__ taps2,
                                            const float2 (&hreg)[TAPS_IN_REGS ? TM : 1], int cp, int r0,
                                            int T, float4 (&acc)[L]) {
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (TM <= 16 && !(Src::kRing && IN != IN_CF32 && L >= PPF_PACKED_MIN_L)) {
        // raw-sample-outer order: all TM taps live in registers, one sample live
        // (scalar FMAs: faster than the packed form below when the samples come
        // from global memory, for fp32 samples and for segments of 2 outputs)
        float2 h[TM];
#pragma unroll
        for (int t = 0; t < TM; ++t) {
            if constexpr (TAPS_IN_REGS) h[t] = hreg[t];
            else h[t] = __ldg(taps2 + t * PAIRS + cp);
        }
        auto run = [&](auto inside_tag) {
            constexpr bool INSIDE = decltype(inside_tag)::value != 0;
#pragma unroll
            for (int i = 0; i < L + TM - 1; ++i) {
                if (i < L + T - 1) {
                    const float4 x = INSIDE ? src.load_inside(r0 + i) : src.load(r0 + i);
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
        };
        if (src.inside(r0, L + T - 1)) run(ic<1>{});
        else run(ic<0>{});
    } else if constexpr (TM <= 16) {
        // samples staged in shared memory, 8/16-bit input, segments of >= 4
        // outputs: packed FMAs on channel pairs -- accumulators (re0, re1) and (im0, im1), taps
        // (h[2cp], h[2cp+1]) as loaded, samples converted straight into pairs
        unsigned long long hp[TM];
#pragma unroll
        for (int t = 0; t < TM; ++t) {
            const float2 h = TAPS_IN_REGS ? hreg[t < (TAPS_IN_REGS ? TM : 1) ? t : 0] : __ldg(taps2 + t * PAIRS + cp);
            hp[t] = pk2(h.x, h.y);
        }
        unsigned long long ar[L], ai[L];
#pragma unroll
        for (int j = 0; j < L; ++j) ar[j] = ai[j] = 0ull;
        // a segment wholly inside the stream loads without per-sample bounds checks
        auto run = [&](auto inside_tag) {
            constexpr bool INSIDE = decltype(inside_tag)::value != 0;
#pragma unroll
            for (int i = 0; i < L + TM - 1; ++i) {
                if (i < L + T - 1) {
                    const float4 x = INSIDE ? src.load_inside(r0 + i) : src.load(r0 + i);
                    const unsigned long long xr = pk2(x.x, x.z), xi = pk2(x.y, x.w);
#pragma unroll
                    for (int j = 0; j < L; ++j) {
                        const int t = i - j;
                        if (t >= 0 && t < TM) {
                            if (IN != IN_CF32 || t < T) {     // fp32: keep inf/NaN out of unrelated outputs
                                ffma2(ar[j], hp[t], xr);       // taps t >= T are zero
                                ffma2(ai[j], hp[t], xi);
                            }
                        }
                    }
                }
            }
        };
        if (src.inside(r0, L + T - 1)) run(ic<1>{});
        else run(ic<0>{});
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const float2 a = upk2(ar[j]), b = upk2(ai[j]);
            acc[j] = make_float4(a.x, b.x, a.y, b.y);
        }
    } else {
        // Large T (T is a runtime bound); packed (re, im) x (h, h) FMAs; a
        // segment wholly inside the stream loads without per-sample bounds
        // checks.  Two orders, chosen per shape by measurement:
        //  * CHUNK (8/16-bit input, C <= 512): the taps in chunks of K held in
        //    registers; for each chunk the raw-sample-outer order of the small-T
        //    path over the L+K-1 rows it needs -- a tap is loaded once per
        //    segment and serves L outputs (rows are re-read per chunk: cheap
        //    for narrow samples);
        //  * otherwise tap-outer with a circular window of L samples (slot
        //    (i mod L) holds raw row r0+i; after tap t the sample r0+t is dead
        //    and its slot is refilled with r0+t+L, L taps before it is needed).
        constexpr int K = 8;
        unsigned long long ap[L][2];
#pragma unroll
        for (int j = 0; j < L; ++j) ap[j][0] = ap[j][1] = 0ull;
        auto run = [&](auto inside_tag) {
            constexpr bool INSIDE = decltype(inside_tag)::value != 0;
            if constexpr (CHUNK) {
#pragma unroll 1
                for (int tc = 0; tc < T; tc += K) {
                    unsigned long long h0[K], h1[K];
#pragma unroll
                    for (int tt = 0; tt < K; ++tt) {
                        const float2 h = (tc + tt < T) ? __ldg(taps2 + (tc + tt) * PAIRS + cp) : make_float2(0.f, 0.f);
                        h0[tt] = pk2(h.x, h.x);
                        h1[tt] = pk2(h.y, h.y);
                    }
#pragma unroll
                    for (int i = 0; i < L + K - 1; ++i) {
                        if (tc + i < L + T - 1) {            // rows past the segment's last tap are not needed
                            const float4 x = INSIDE ? src.load_inside(r0 + tc + i) : src.load(r0 + tc + i);
                            const unsigned long long x01 = pk2(x.x, x.y), x23 = pk2(x.z, x.w);
#pragma unroll
                            for (int j = 0; j < L; ++j) {
                                const int tt = i - j;
                                if (tt >= 0 && tt < K) {
                                    if (IN != IN_CF32 || tc + tt < T) {   // fp32: keep inf/NaN out of unrelated outputs
                                        ffma2(ap[j][0], h0[tt], x01);
                                        ffma2(ap[j][1], h1[tt], x23);
                                    }
                                }
                            }
                        }
                    }
                }
            } else {
                auto ld = [&](int r) { return INSIDE ? src.load_inside(r) : src.load(r); };
                float4 xw[L];
#pragma unroll
                for (int i = 0; i < L; ++i) xw[i] = ld(r0 + i);
#pragma unroll 1
                for (int tb = 0; tb < T; tb += L) {
#pragma unroll
                    for (int u = 0; u < L; ++u) {
                        const int t = tb + u;
                        if (t < T) {
                            const float2 h = __ldg(taps2 + t * PAIRS + cp);
                            const unsigned long long h0 = pk2(h.x, h.x), h1 = pk2(h.y, h.y);
#pragma unroll
                            for (int j = 0; j < L; ++j) {
                                const float4 x = xw[(j + u) % L];
                                ffma2(ap[j][0], h0, pk2(x.x, x.y));
                                ffma2(ap[j][1], h1, pk2(x.z, x.w));
                            }
                            if (t + 1 < T) xw[u] = ld(r0 + t + L);
                        }
                    }
                }
            }
        };
        if (src.inside(r0, L + T - 1)) run(ic<1>{});
        else run(ic<0>{});
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const float2 a = upk2(ap[j][0]), b = upk2(ap[j][1]);
            acc[j] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// The FIR + DFT of output batches [lo, hi) of one stream (in/out already
// offset to the stream), by the whole CTA, using `smem`.  Returns false when
// a bounded wait gave up (the status word is then set).  Safe to call again
// for another range (the tile loop of the multi-beam kernel).
template <int C, int TM, int IN, int OUT, int NTO = 0, class GRP = CtaGroup>
__device__ __forceinline__ bool fwd_range(const FwdArgs& args, const void* in, void* out, long long lo,
                                          long long hi, unsigned char* smem) {
    using S = FwdShape<C, TM, IN, NTO>;
    constexpr int NT = S::NT, B = S::B, L = S::L, NS = S::NS;
    constexpr int NST = fft_stages(C);
    constexpr bool RING = S::RING;
    float2* ybuf = reinterpret_cast<float2*>(smem);
    float2* ybuf2 = reinterpret_cast<float2*>(smem + S::YBYTES);        // PINGPONG only
    float2* tw_s = reinterpret_cast<float2*>(smem + S::YB);
    unsigned char* ring = smem + S::RING_OFF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + NS * S::SLOTB);   // NS + 1 barriers
    volatile int* sflag = reinterpret_cast<volatile int*>(bars + NS + 1);

    const int tid = GRP::tid();
    const long long n_spectra = args.n_spectra;
    const int T = args.T;
    const long long n_raw = n_spectra + T - 1;
    const long long nb = hi - lo;
    if (nb <= 0) return true;
    GRP::sync();   // the previous range of this CTA is done with shared memory
    const float2* tws = args.tw;
    if constexpr (S::TW_SMEM) {
        for (int i = tid; i < tw_size(C); i += NT) tw_s[i] = args.tw[i];
        tws = tw_s;
    }
    const float2* taps2 = reinterpret_cast<const float2*>(args.taps);   // [t][pair]
    float2 hreg[S::TAPS_IN_REGS ? TM : 1];
    if constexpr (S::TAPS_IN_REGS) {
#pragma unroll
        for (int t = 0; t < TM; ++t) hreg[t] = __ldg(taps2 + t * S::PAIRS + tid % S::PAIRS);
    }

    // ------------------------------------------------------- ring set-up
    // Relative batch j (0 <= j <= nb; j == nb is the halo-only batch) has
    // raw rows [(lo+j)*B, (lo+j)*B + B) clipped to the stream.
    auto rows_of = [&](long long j) -> long long {
        const long long r = n_raw - (lo + j) * B;
        return r <= 0 ? 0 : (r < B ? r : B);
    };
    // last relative batch the FIRs read: the halo of the range's last batch
    // ends in batch nb-1 + ceil((T-1)/B) (rows past the stream are not copied)
    const long long last_needed = nb - 1 + (T - 1 + B - 1) / B;
    long long issued = 0, waited = 0;                        // meaningful in thread 0 only
    auto issue = [&](long long j) {
        const long long rows = rows_of(j);
        if (rows > 0) {
            uint64_t* bar = &bars[j % NS];
            const uint32_t bytes = (uint32_t)(rows * C * S::BIN);
            mbar_expect_tx(bar, bytes);
            const unsigned char* src = static_cast<const unsigned char*>(in) + (size_t)(lo + j) * B * C * S::BIN;
            if constexpr (PPF_TMA_EVICT_FIRST) tma_load_1d_once(ring + (j % NS) * S::SLOTB, src, bytes, bar);
            else tma_load_1d(ring + (j % NS) * S::SLOTB, src, bytes, bar);
        }
    };
    auto wait_upto = [&](long long j) -> bool {            // thread 0: batches < issued only
        bool ok = true;
        for (; waited <= j && waited < issued; ++waited) {
            if (rows_of(waited) > 0)
                ok = ok && mbar_wait_bounded(&bars[waited % NS], (uint32_t)((waited / NS) & 1), kWaitLimitNs);
        }
        return ok;
    };
    if constexpr (RING) {
        if (tid == 0) {
            for (int i = 0; i <= NS; ++i) mbar_init(&bars[i], 1);
            fence_mbar_init();
            *sflag = 0;
        }
        GRP::sync();
        if (tid == 0) {
            fence_proxy_async_smem();   // the slots were last read by the previous range's FIR
            for (; issued < NS && issued <= last_needed; ++issued) issue(issued);
        }
    }
    GRP::sync();

    for (long long k = 0; k < nb; ++k) {
        const long long sb = (lo + k) * B;          // first output spectrum of the batch
        if constexpr (RING) {
            if (tid == 0) {
                bool ok = wait_upto(k + (T - 1 + B - 1) / B);
                if (k == 0 && (args.flags & FWD_INJECT_TIMEOUT))  // a barrier nothing arrives on
                    ok = ok && mbar_wait_bounded(&bars[NS], 0, kInjectedWaitNs);
                if (!ok) {
                    // give up: let every copy in flight land, then report
                    for (; waited < issued; ++waited)
                        if (rows_of(waited) > 0)
                            mbar_wait_bounded(&bars[waited % NS], (uint32_t)((waited / NS) & 1), kWaitLimitNs);
                    atomicExch(args.err, 1);
                    *sflag = 1;
                }
            }
            GRP::sync();
            if (*sflag) return false;
        } else {
            if (tid == 0 && k + 2 < nb) {           // warm L2 two batches ahead
                const long long r0 = (sb + 2 * B), rows = (n_raw - r0 < B) ? n_raw - r0 : B;
                if (rows > 0)
                    tma_prefetch_l2(static_cast<const unsigned char*>(in) + (size_t)r0 * C * S::BIN,
                                    (uint32_t)(rows * C * S::BIN));
            }
        }
        // ---------------------------------------------------------- FIR
#pragma unroll 1
        for (int f = 0; f < S::FPT; ++f) {
            const int item = tid + f * NT;
            if (!S::FIR_EXACT && item >= S::FIR_ITEMS) break;
            const int cp = item % S::PAIRS, g = item / S::PAIRS;
            RawSrc<C, IN, RING, B, S::HS> src;
            if constexpr (RING) {
#pragma unroll
                for (int h = 0; h <= S::HS; ++h) src.sl[h] = ring + ((k + h) % NS) * S::SLOTB + 2 * cp * S::BIN;
            } else {
                src.in = in;
                src.row0 = sb;
                src.n_raw = n_raw;
                src.cp = cp;
            }
            float4 acc[L];
            fir_segment<TM, IN, L, S::PAIRS, S::TAPS_IN_REGS, S::CHUNK>(src, taps2, hreg, cp, S::G == 1 ? 0 : g * L,
                                                                        T, acc);
#pragma unroll
            for (int j = 0; j < L; ++j)
                *reinterpret_cast<float4*>(ybuf + (g * L + j) * C + 2 * cp) = acc[j];
        }
        GRP::sync();
        if constexpr (RING) {
            // slot k is free: refill it with batch k+NS
            if (tid == 0 && issued <= last_needed && issued == k + NS) {
                fence_proxy_async_smem();
                issue(issued);
                ++issued;
            }
        }
        // ---------------------------------------------------------- FFT
        if constexpr (S::PINGPONG) {
            // stage p reads buffer p & 1 and writes buffer (p + 1) & 1; the last
            // stage's reads are ordered before the next batch's FIR writes by the
            // barrier after the ring wait, or by the one below without a ring
            static_for<NST>([&](auto p) {
                constexpr int P = decltype(p)::value;
                fft_stage<C, B, NT, P, OUT, S::TW_SMEM, 0, false, false, 0, GRP, true>(
                    (P & 1) ? ybuf2 : ybuf, tws, out, sb, 0, n_spectra, (P & 1) ? ybuf : ybuf2);
            });
            if constexpr (!RING) GRP::sync();
        } else {
            static_for<NST>([&](auto p) {
                fft_stage<C, B, NT, decltype(p)::value, OUT, S::TW_SMEM, 0, false, false, 0, GRP>(ybuf, tws, out, sb, 0,
                                                                                                  n_spectra);
            });
        }
    }
    if constexpr (RING) {
        // every copy of the range has landed (thread 0 waited for each):
        // retire the barriers, the next range of this CTA initialises them anew
        if (tid == 0)
            for (int i = 0; i <= NS; ++i) mbar_inval(&bars[i]);
    }
    return true;
}

// The batches of all streams form one sequence (stream-major, nbt per stream);
// work unit `unit` of `n_units` owns the equal contiguous share [u0, u1),
// which it walks as segments [lo, hi) of single streams.
struct BatchShare {
    long long nbt, u, u1;
    __device__ __forceinline__ BatchShare(long long nbt_, long long n_streams, int unit, int n_units)
        : nbt(nbt_), u((long long)unit * (nbt_ * n_streams) / n_units),
          u1((long long)(unit + 1) * (nbt_ * n_streams) / n_units) {}
    // next segment: stream and batch range; false when the share is done
    __device__ __forceinline__ bool next(long long& strm, long long& lo, long long& hi) {
        if (u >= u1) return false;
        strm = u / nbt;
        lo = u - strm * nbt;
        hi = (u1 - strm * nbt < nbt) ? u1 - strm * nbt : nbt;
        u = strm * nbt + hi;
        return true;
    }
};

template <int C, int TM, int IN, int OUT>
__global__ void __launch_bounds__(FwdShape<C, TM, IN>::NT, FwdShape<C, TM, IN>::NT == 256 ? 2 : 1)
pfb_fwd_kernel(FwdArgs args) {
    using S = FwdShape<C, TM, IN>;
    extern __shared__ __align__(128) unsigned char smem[];
    // the CTA's share of the batches: raw spectra stream through the CTA once
    BatchShare share((args.n_spectra + S::B - 1) / S::B, args.n_streams, blockIdx.x, gridDim.x);
    long long strm, lo, hi;
    while (share.next(strm, lo, hi)) {
        const void* in = static_cast<const unsigned char*>(args.in) + (size_t)strm * args.in_stride * S::BIN;
        void* out = static_cast<unsigned char*>(args.out) + (size_t)strm * args.out_stride * (OUT == OUT_CF32 ? 8 : 4);
        if (!fwd_range<C, TM, IN, OUT>(args, in, out, lo, hi, smem)) return;
    }
}

// Host side: shape + launch of one instantiation.
struct FwdInfo {
    int threads, batch, smem, stages, tap_bucket, variant;
    const void* fn;
    int cluster;     // CTAs per thread-block cluster (0: no cluster)
};

}  // namespace ppf

#include "ppf_fwd_carry.cuh"
#include "ppf_fwd_cluster.cuh"
#include "ppf_fwd_push.cuh"
#include "ppf_fwd_longtap.cuh"

// Selection switches.  The push-exchange cluster kernel (C = 2048/4096, int8)
// passes every parity test but measured slower than the cluster and generic
// kernels it would replace, so it is compiled only when enabled.  The
// long-tap kernel (T = 17..64, C <= 512) is the default for those shapes
// (1.1 - 1.7x the generic kernel).
#ifndef PPF_NO_PUSH
#define PPF_NO_PUSH 1
#endif
#ifndef PPF_NO_LONGTAP
#define PPF_NO_LONGTAP 0
#endif

namespace ppf {

// The carry kernel where it fits, except at C = 1024 with 9-16 taps: its 512
// threads get at most 128 registers for a carried state estimated at 192,
// and the generic kernel's ring (two CTAs per SM) measured faster there
// (int8 T = 16: 247 vs 203 GS/s).  The multi-beam kernel and the FIR-only
// ablation keep the carry body for those shapes.
template <int C, int TM, int IN>
constexpr bool carry_preferred() {
    return CarryShape<C, TM, IN>::OK && !(C == 1024 && TM > 8);
}

template <int C, int TM, int IN, int OUT>
inline FwdInfo fwd_info() {
    if constexpr (carry_preferred<C, TM, IN>()) {
        using S = CarryShape<C, TM, IN>;
        return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM, 1 | (S::TW_SMEM ? 2 : 0) | 4,
                       reinterpret_cast<const void*>(&pfb_fwd_carry_kernel<C, TM, IN, OUT>), 0};
    } else if constexpr (PushShape<C, TM, IN>::OK && !PPF_NO_PUSH) {
        using S = PushShape<C, TM, IN>;
        return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM, 1 | 2 | 4 | 16 | 32,
                       reinterpret_cast<const void*>(&pfb_fwd_push_kernel<C, TM, IN, OUT>), S::Q};
    } else if constexpr (ClusterShape<C, TM, IN>::OK) {
        using S = ClusterShape<C, TM, IN>;
        return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM, 1 | (S::TW_SMEM ? 2 : 0) | 4 | 16,
                       reinterpret_cast<const void*>(&pfb_fwd_cluster_kernel<C, TM, IN, OUT>), S::Q};
    } else if constexpr (TM == 64 && LongShape<C, IN>::OK && !PPF_NO_LONGTAP) {
        using S = LongShape<C, IN>;
        return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM, 1 | 2 | 64,
                       reinterpret_cast<const void*>(&pfb_fwd_longtap_kernel<C, IN, OUT>), 0};
    } else {
        using S = FwdShape<C, TM, IN>;
        return FwdInfo{S::NT, S::B, S::SMEM, fft_stages(C), TM, (S::RING ? 1 : 0) | (S::TW_SMEM ? 2 : 0),
                       reinterpret_cast<const void*>(&pfb_fwd_kernel<C, TM, IN, OUT>), 0};
    }
}

// grid: CTAs (a multiple of the cluster size for cluster kernels).
template <int C, int TM, int IN, int OUT>
inline cudaError_t fwd_launch(const FwdArgs& a, int grid, cudaStream_t st) {
    if constexpr (carry_preferred<C, TM, IN>()) {
        using S = CarryShape<C, TM, IN>;
        pfb_fwd_carry_kernel<C, TM, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    } else if constexpr (PushShape<C, TM, IN>::OK && !PPF_NO_PUSH) {
        using S = PushShape<C, TM, IN>;
        pfb_fwd_push_kernel<C, TM, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    } else if constexpr (ClusterShape<C, TM, IN>::OK) {
        using S = ClusterShape<C, TM, IN>;
        pfb_fwd_cluster_kernel<C, TM, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    } else if constexpr (TM == 64 && LongShape<C, IN>::OK && !PPF_NO_LONGTAP) {
        using S = LongShape<C, IN>;
        pfb_fwd_longtap_kernel<C, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    } else {
        using S = FwdShape<C, TM, IN>;
        pfb_fwd_kernel<C, TM, IN, OUT><<<grid, S::NT, S::SMEM, st>>>(a);
    }
    return cudaPeekAtLastError();
}

// FIR-only ablation kernels (carry shapes only), output complex FP32 rows.
template <int C, int TM, int IN>
inline bool fir_info(FwdInfo* i) {
    if constexpr (CarryShape<C, TM, IN>::OK) {
        using S = CarryShape<C, TM, IN>;
        *i = FwdInfo{S::NT, S::B, S::SMEM, 0, TM, 8,
                     reinterpret_cast<const void*>(&pfb_fwd_carry_kernel<C, TM, IN, OUT_CF32, true>), 0};
        return true;
    } else {
        return false;
    }
}

template <int C, int TM, int IN>
inline cudaError_t fir_launch(const FwdArgs& a, int grid, cudaStream_t st) {
    if constexpr (CarryShape<C, TM, IN>::OK) {
        using S = CarryShape<C, TM, IN>;
        pfb_fwd_carry_kernel<C, TM, IN, OUT_CF32, true><<<grid, S::NT, S::SMEM, st>>>(a);
        return cudaPeekAtLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// Twiddle table contents (host, FP64 -> FP32): stage p < P-1 holds
// W_{N_p}^{b k} = exp(-2 pi i b k / N_p), k = 1 .. R_p-1, at
// [tw_offset(p) + (k-1)*N_{p+1} + b].
// Entries of the plan's twiddle table for C.
constexpr int tw_total_float2s(int C) { return tw_size(C); }

template <int C>
inline void fill_twiddles(float2* host) {
    for (int p = 0; p + 1 < fft_stages(C); ++p) {
        const int NP = fft_n(C, p), R = fft_radix(C, p), NN = NP / R;
        for (int k = 1; k < R; ++k)
            for (int b = 0; b < NN; ++b) {
                const long e = (long)b * k % NP;
                host[tw_offset(C, p) + (k - 1) * NN + b] =
                    make_float2((float)cos2pi(e, NP), (float)(-sin2pi(e, NP)));
            }
    }
}

}  // namespace ppf
