// ppf_device.cuh -- device building blocks of the fused PFB kernels (sm_103a).
//
// * compile-time twiddles: cos/sin of 2*pi*k/N evaluated in FP64 by a Taylor
//   series at compile time and rounded once to FP32;
// * in-register C-point DFT building block dft_reg<N> (radix-4 / radix-2
//   decimation in frequency, natural order in and out);
// * loads of a channel pair for each input type with the int -> FP32
//   conversion fused in;
// * streaming stores of complex FP32 / FP16 output.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace ppf {

// ---------------------------------------------------------------- utilities

template <int... Is> struct iseq {};
template <int N, int... Is> struct make_iseq_t : make_iseq_t<N - 1, N - 1, Is...> {};
template <int... Is> struct make_iseq_t<0, Is...> { using type = iseq<Is...>; };
template <int I> struct ic { static constexpr int value = I; };

// static_for<N>(f): calls f(ic<0>{}), ..., f(ic<N-1>{}) with compile-time indices.
template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, iseq<Is...>) {
    (f(ic<Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, typename make_iseq_t<N>::type{});
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ------------------------------------------------------ compile-time trig
// sin(x) for x in [0, pi/4] by its Taylor series, enough terms for FP64.
constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 14; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 14; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
constexpr double kPi = 3.14159265358979323846264338327950288;

// cos and sin of 2*pi*k/n for integers, with the octant reduction done on
// the integer 8k mod 8n so the Taylor argument stays in [0, pi/4].
constexpr double cos2pi(long k, long n) {
    k %= n; if (k < 0) k += n;
    long e = 8 * k;               // angle = (2 pi / (8n)) * e
    long oct = e / n;             // octant 0..7
    long r = e - oct * n;         // remainder: angle within octant = 2 pi r / (8 n)
    double a = 2.0 * kPi * (double)r / (8.0 * (double)n);   // [0, pi/4)
    double b = kPi / 4.0 - a;                                // for odd octants
    switch (oct) {
        case 0: return taylor_cos(a);
        case 1: return taylor_sin(b);
        case 2: return -taylor_sin(a);
        case 3: return -taylor_cos(b);
        case 4: return -taylor_cos(a);
        case 5: return -taylor_sin(b);
        case 6: return taylor_sin(a);
        default: return taylor_cos(b);
    }
}
constexpr double sin2pi(long k, long n) { return cos2pi(4 * k - n, 4 * n); }  // sin x = cos(x - pi/2)

// W_N^m = exp(-2 pi i m / N) as FP32 constants.
template <int M, int N> struct Tw {
    static constexpr float re = (float)cos2pi(M, N);
    static constexpr float im = (float)(-sin2pi(M, N));
};

// ---------------------------------------------------------- complex helpers
// Complex add/sub use the packed FP32 pair instructions of sm_100+ (one
// instruction for re and im); everything else is scalar FP32.
__device__ __forceinline__ unsigned long long as_pair(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 from_pair(unsigned long long v) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(v));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#ifndef PPF_NO_F32X2
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_pair(a)), "l"(as_pair(b)));
    return from_pair(r);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
#ifndef PPF_NO_F32X2
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_pair(a)), "l"(as_pair(b)));
    return from_pair(r);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
// a * w for a runtime twiddle w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * (-i)
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// a * W_N^M with the trivial cases folded at compile time.
template <int M, int N>
__device__ __forceinline__ float2 cmul_tw(float2 a) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (4 * m == N) {                 // -i
        return make_float2(a.y, -a.x);
    } else if constexpr (2 * m == N) {                 // -1
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * m == 3 * N) {             // +i
        return make_float2(-a.y, a.x);
    } else if constexpr (8 * m == N) {                 // (1 - i)/sqrt2: (x + y) r, (y - x) r
        constexpr float r = Tw<1, 8>::re;
        const float t = a.y * r;                      // 3 instructions: y r, then x r +/- y r fused
        return make_float2(fmaf(a.x, r, t), fmaf(-a.x, r, t));
    } else if constexpr (8 * m == 3 * N) {             // (-1 - i)/sqrt2: (y - x) r, -(x + y) r
        constexpr float r = Tw<1, 8>::re;
        const float t = a.y * r;
        return make_float2(fmaf(-a.x, r, t), fmaf(-a.x, r, -t));
    } else {
        constexpr float wr = Tw<m, N>::re, wi = Tw<m, N>::im;
        return make_float2(fmaf(a.x, wr, -a.y * wi), fmaf(a.x, wi, a.y * wr));
    }
}

// ------------------------------------------------------- in-register DFT
constexpr int bitrev(int k, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (k & 1); k >>= 1; }
    return r;
}

// One radix-4 DIF butterfly group over a block of length LEN = 4*S at BASE,
// element j (0 <= J < S): two fused radix-2 DIF stages.
template <int LEN, int BASE, int J, int N>
__device__ __forceinline__ void r4_bfly(float2 (&v)[N]) {
    constexpr int S = LEN / 4;
    float2 a0 = v[BASE + J], a1 = v[BASE + J + S], a2 = v[BASE + J + 2 * S], a3 = v[BASE + J + 3 * S];
    float2 p = cadd(a0, a2), q = csub(a0, a2);
    float2 r = cadd(a1, a3), d = csub(a1, a3);
    // q + (-i) d and q - (-i) d: the swap of d's parts folds into scalar adds
    const float2 u = make_float2(q.x + d.y, q.y - d.x), w = make_float2(q.x - d.y, q.y + d.x);
    v[BASE + J] = cadd(p, r);
    v[BASE + J + S] = cmul_tw<2 * J, LEN>(csub(p, r));
    v[BASE + J + 2 * S] = cmul_tw<J, LEN>(u);
    v[BASE + J + 3 * S] = cmul_tw<3 * J, LEN>(w);
}

template <int LEN, int N>
__device__ __forceinline__ void dif_stage(float2 (&v)[N]) {
    if constexpr (LEN >= 4) {
        static_for<N / LEN>([&](auto b) {
            static_for<LEN / 4>([&](auto j) { r4_bfly<LEN, decltype(b)::value * LEN, decltype(j)::value>(v); });
        });
        dif_stage<LEN / 4>(v);
    } else if constexpr (LEN == 2) {
        static_for<N / 2>([&](auto b) {
            constexpr int i = decltype(b)::value * 2;
            float2 a0 = v[i], a1 = v[i + 1];
            v[i] = cadd(a0, a1);
            v[i + 1] = csub(a0, a1);
        });
    }
}

// dft_reg<N>: v[k] <- sum_n v[n] exp(-2 pi i n k / N), natural order in/out.
// N a power of two, or 3 (first stage of the C = 3 * 2^k transforms).
template <int N>
__device__ __forceinline__ void dft_reg(float2 (&v)[N]) {
    static_assert(is_pow2(N) || N == 3, "radix must be a power of two or 3");
    if constexpr (N == 3) {
        // W = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
        constexpr float h = 0.866025403784438646763723170752936183f;   // sqrt(3)/2
        const float2 s = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
        const float2 d = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
        const float2 t = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
        const float2 u = make_float2(h * d.y, -h * d.x);                  // -i sqrt(3)/2 d
        v[0] = make_float2(v[0].x + s.x, v[0].y + s.y);
        v[1] = make_float2(t.x + u.x, t.y + u.y);
        v[2] = make_float2(t.x - u.x, t.y - u.y);
    } else if constexpr (N > 1) {
        dif_stage<N>(v);
        float2 t[N];
        static_for<N>([&](auto k) { t[decltype(k)::value] = v[bitrev(decltype(k)::value, ilog2(N))]; });
        static_for<N>([&](auto k) { v[decltype(k)::value] = t[decltype(k)::value]; });
    }
}

// ------------------------------------------------------------ input loads
// One channel pair (c, c+1) of one raw spectrum: 4 floats (re0, im0, re1, im1).
enum InType { IN_CI8 = 0, IN_CI16 = 1, IN_CF32 = 2 };
enum OutType { OUT_CF32 = 0, OUT_CF16 = 1 };

template <int IN> struct InTraits;
template <> struct InTraits<IN_CI8>  { static constexpr int bytes = 2; };
template <> struct InTraits<IN_CI16> { static constexpr int bytes = 4; };
template <> struct InTraits<IN_CF32> { static constexpr int bytes = 8; };

__device__ __forceinline__ float4 cvt_ci8x2(uint32_t w) {
    return make_float4((float)(int8_t)(w & 0xff), (float)(int8_t)((w >> 8) & 0xff),
                       (float)(int8_t)((w >> 16) & 0xff), (float)(int8_t)(w >> 24));
}
__device__ __forceinline__ float4 cvt_ci16x2(uint2 w) {
    return make_float4((float)(int16_t)(w.x & 0xffff), (float)(int16_t)(w.x >> 16),
                       (float)(int16_t)(w.y & 0xffff), (float)(int16_t)(w.y >> 16));
}

// Load the pair at sample offset `off` (even) through the read-only path.
template <int IN>
__device__ __forceinline__ float4 load_pair_global(const void* __restrict__ base, long long off) {
    if constexpr (IN == IN_CI8) {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(static_cast<const int8_t*>(base) + 2 * off);
        return cvt_ci8x2(__ldg(p));
    } else if constexpr (IN == IN_CI16) {
        const uint2* p = reinterpret_cast<const uint2*>(static_cast<const int16_t*>(base) + 2 * off);
        return cvt_ci16x2(__ldg(p));
    } else {
        const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(base) + 2 * off);
        return __ldg(p);
    }
}

// ------------------------------------------------------- packed FP32 pairs
// (re, im) or two lanes of FP32 as one 64-bit register pair
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
// d += a * b, two FP32 lanes per instruction
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// ---------------------------------------------------------------- stores
#ifndef PPF_STORE_CS
#define PPF_STORE_CS 1
#endif
template <int OUT>
__device__ __forceinline__ void store_out(void* __restrict__ base, long long idx, float2 v) {
    if constexpr (OUT == OUT_CF32) {
        if constexpr (PPF_STORE_CS) __stcs(reinterpret_cast<float2*>(base) + idx, v);
        else reinterpret_cast<float2*>(base)[idx] = v;
    } else {
        __half2 h = __float22half2_rn(v);
        if constexpr (PPF_STORE_CS) __stcs(reinterpret_cast<unsigned int*>(base) + idx, *reinterpret_cast<unsigned int*>(&h));
        else reinterpret_cast<unsigned int*>(base)[idx] = *reinterpret_cast<unsigned int*>(&h);
    }
}

}  // namespace ppf

namespace ppf {

// ------------------------------------------------ TMA bulk copies, mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Retire a barrier whose operations have all completed, before its memory is
// initialised again (the next range of a kernel that re-initialises per range).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Generic-proxy accesses to shared memory before this fence are ordered
// before later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Plain arrival (release at CTA scope) on a barrier of this CTA.
__device__ __forceinline__ void mbar_arrive_cta(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of `bar` to complete; gives up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}
// 1-D bulk copy global -> shared completing on `bar` (bytes multiple of 16,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// The same copy with an L2 evict-first policy for the source lines (data
// read exactly once, so it need not displace the output lines in L2).
__device__ __forceinline__ void tma_load_1d_once(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
// Hint: bring a global range into L2 ahead of its use (bytes multiple of 16).
__device__ __forceinline__ void tma_prefetch_l2(const void* src_gmem, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src_gmem), "r"(bytes) : "memory");
}

// Asynchronous 4/8/16-byte copy global -> shared (the thread's own staging
// slot), committed in groups; wait_group<N> returns once at most N of the
// thread's most recent groups are still in flight.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src_gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Bulk copy shared -> global through the async proxy (bulk-group completion).
// dst, src and bytes must be multiples of 16.  The writing threads make their
// shared-memory stores visible to the async proxy (fence_proxy_async_smem)
// and synchronise before one thread issues the copy.
__device__ __forceinline__ void tma_store_1d(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// The source shared memory of every committed bulk store may be overwritten.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// One complex sample (2 floats) at byte address p of shared memory / global memory.
template <int IN>
__device__ __forceinline__ float2 load_one_smem(const unsigned char* p) {
    if constexpr (IN == IN_CI8) {
        const uint32_t w = *reinterpret_cast<const uint16_t*>(p);
        return make_float2((float)(int8_t)(w & 0xff), (float)(int8_t)(w >> 8));
    } else if constexpr (IN == IN_CI16) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
        return make_float2((float)(int16_t)(w & 0xffff), (float)(int16_t)(w >> 16));
    } else {
        return *reinterpret_cast<const float2*>(p);
    }
}
template <int IN>
__device__ __forceinline__ float2 load_one_global(const void* __restrict__ base, long long off) {
    if constexpr (IN == IN_CI8) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned short*>(base) + off);
        return make_float2((float)(int8_t)(w & 0xff), (float)(int8_t)(w >> 8));
    } else if constexpr (IN == IN_CI16) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(base) + off);
        return make_float2((float)(int16_t)(w & 0xffff), (float)(int16_t)(w >> 16));
    } else {
        return __ldg(reinterpret_cast<const float2*>(base) + off);
    }
}

// One channel pair (4 floats) from shared memory at byte address p.
template <int IN>
__device__ __forceinline__ float4 load_pair_smem(const unsigned char* p) {
    if constexpr (IN == IN_CI8) {
        return cvt_ci8x2(*reinterpret_cast<const uint32_t*>(p));
    } else if constexpr (IN == IN_CI16) {
        return cvt_ci16x2(*reinterpret_cast<const uint2*>(p));
    } else {
        return *reinterpret_cast<const float4*>(p);
    }
}

}  // namespace ppf
