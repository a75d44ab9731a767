// ppf_probe.cu -- throughput micro-benchmarks for the measurement of the
// PFB kernels: the rate of integer -> FP32 type conversions (the limit the
// paper reports for low-precision input, Sec. 4.1 Table 3 "bit-conversions",
// measured with its own micro-benchmark) and of scalar and packed (f32x2)
// FP32 fused multiply-adds, the other pipe the FIR and FFT load.
//
// Each probe runs independent dependency chains per thread on every SM and
// is timed with CUDA events; results are operations per second (a packed
// f32x2 FMA counts as two FMAs; a conversion of one value counts as one).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/ppf.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}

__global__ void k_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
    unsigned long long x[kChains];
    const unsigned long long A = pack2(a, a), Bv = pack2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = pack2(threadIdx.x * 1e-3f + c, c * 0.5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(Bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) { float2 v = unpack2(x[c]); s += v.x + v.y; }
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// int8 -> FP32 with the compiler's conversion (cvt.rn.f32.s8 on extracted bytes)
__global__ void k_cvt_s8(float* out, int iters, uint32_t seed) {
    uint32_t w[kChains];
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) { w[c] = seed * (threadIdx.x + 1) + c; acc[c] = 0.f; }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t v = w[c];
            acc[c] += (float)(int8_t)(v & 0xff) + (float)(int8_t)((v >> 8) & 0xff)
                    + (float)(int8_t)((v >> 16) & 0xff) + (float)(int8_t)(v >> 24);
            w[c] = v + 0x01010101u;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// int8 -> FP32 by the exponent-bias ("magic number") method, a standard
// integer-to-float technique (H. S. Warren, Hacker's Delight, 2nd ed., ch. 17,
// converting between integer and floating point): the biased byte (b ^ 0x80)
// is placed in the low mantissa bits of 2^23 (0x4B000000) with a byte
// permute, and 2^23 + 128 is subtracted; exact for all 256 byte values.
__device__ __forceinline__ float i8_bias(uint32_t wx, uint32_t sel) {
    return __int_as_float(__byte_perm(wx, 0x4B000000u, sel)) - 8388736.0f;
}
__global__ void k_cvt_s8_bias(float* out, int iters, uint32_t seed) {
    uint32_t w[kChains];
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) { w[c] = seed * (threadIdx.x + 1) + c; acc[c] = 0.f; }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t v = w[c] ^ 0x80808080u;
            acc[c] += i8_bias(v, 0x7440u) + i8_bias(v, 0x7441u) + i8_bias(v, 0x7442u) + i8_bias(v, 0x7443u);
            w[c] = w[c] + 0x01010101u;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void k_cvt_s16(float* out, int iters, uint32_t seed) {
    uint32_t w[kChains];
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) { w[c] = seed * (threadIdx.x + 1) + c; acc[c] = 0.f; }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t v = w[c];
            acc[c] += (float)(int16_t)(v & 0xffff) + (float)(int16_t)(v >> 16);
            w[c] = v + 0x00010001u;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// Streaming kernel with a chosen read:write ratio: every thread reads 16-byte
// vectors from `in` and writes `ratio` 16-byte vectors to `out` (the traffic
// mix of a PFB with narrow input and wide output, e.g. int8 in, complex FP32
// out = 1:4).  Grid-stride, coalesced, streaming stores.
__global__ void k_stream(const uint4* __restrict__ in, uint4* __restrict__ out, long long n_in, int ratio) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += stride) {
        const uint4 v = __ldcs(in + i);
        for (int r = 0; r < ratio; ++r) {
            uint4 w = v;
            w.x += r;
            __stcs(out + (size_t)r * n_in + i, w);
        }
    }
}

template <class F>
double time_kernel(F launch, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms * 1e-3 / reps;
}

}  // namespace

// Rates in operations per second, written to rates[0..n):
//   0 scalar FP32 FMA, 1 packed f32x2 FMA (2 per instruction), 2 int8->FP32
//   conversions (compiler cvt), 3 int8->FP32 by exponent bias, 4 int16->FP32.
// Synchronous; uses the legacy default stream.
extern "C" ppf_status ppf_probe_rates(double* rates, int n) {
    if (rates == nullptr || n < 1) return PPF_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PPF_ERR_CUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * sms * 8) != cudaSuccess) return PPF_ERR_OUT_OF_MEMORY;
    const int grid = sms * 8, block = 256, iters = 4096, reps = 5;
    const double threads = (double)grid * block;
    double r[5];
    r[0] = threads * iters * kChains / time_kernel([&] { k_ffma<<<grid, block>>>(out, iters, 0.999f, 1e-3f); }, reps);
    r[1] = 2.0 * threads * iters * kChains / time_kernel([&] { k_ffma2<<<grid, block>>>(out, iters, 0.999f, 1e-3f); }, reps);
    r[2] = 4.0 * threads * iters * kChains / time_kernel([&] { k_cvt_s8<<<grid, block>>>(out, iters, 7u); }, reps);
    r[3] = 4.0 * threads * iters * kChains / time_kernel([&] { k_cvt_s8_bias<<<grid, block>>>(out, iters, 7u); }, reps);
    r[4] = 2.0 * threads * iters * kChains / time_kernel([&] { k_cvt_s16<<<grid, block>>>(out, iters, 7u); }, reps);
    cudaError_t e = cudaGetLastError();
    cudaFree(out);
    if (e != cudaSuccess) return PPF_ERR_CUDA;
    for (int i = 0; i < n && i < 5; ++i) rates[i] = r[i];
    return PPF_OK;
}

// Achievable DRAM bandwidth (bytes read + written per second) of a streaming
// kernel that reads in_bytes and writes ratio * in_bytes; synchronous, uses
// caller-provided device buffers (in: in_bytes, out: ratio * in_bytes, both
// 16-byte aligned, in_bytes a multiple of 16).
extern "C" ppf_status ppf_probe_stream(const void* in_dev, void* out_dev, long long in_bytes, int ratio,
                                       double* bytes_per_s) {
    if (in_dev == nullptr || out_dev == nullptr || bytes_per_s == nullptr || in_bytes < 16 || (in_bytes & 15) ||
        ratio < 0 || ratio > 16 || ((reinterpret_cast<uintptr_t>(in_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15))
        return PPF_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PPF_ERR_CUDA;
    const long long n = in_bytes / 16;
    double t = 1e30;
    for (int rep = 0; rep < 3; ++rep)
        t = fmin(t, time_kernel([&] {
            k_stream<<<sms * 4, 512>>>(static_cast<const uint4*>(in_dev), static_cast<uint4*>(out_dev), n, ratio);
        }, 3));
    if (cudaGetLastError() != cudaSuccess) return PPF_ERR_CUDA;
    *bytes_per_s = (double)in_bytes * (1 + ratio) / t;
    return PPF_OK;
}
