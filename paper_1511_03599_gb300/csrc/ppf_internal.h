// ppf_internal.h -- host-side interface between the C ABI and the per-C
// kernel instantiation units (one object per channel count C, built from
// ppf_fwd_inst.cu with -DPPF_C=<C>).
#pragma once

#include <cuda_runtime.h>

#include "../../include/ppf.h"

namespace ppf {

// Record the detail of an error for ppf_last_error_message (calling thread)
// and return the status.
ppf_status set_error(ppf_status s, const char* fmt, ...);

struct FwdArgs;
struct BwdArgs;
struct IdftArgs;
struct AdjFirArgs;
struct AdjCorrArgs;

struct FwdEntry {
    int threads;     // threads per CTA
    int batch;       // output spectra per CTA batch
    int smem;        // dynamic shared memory bytes
    int stages;      // FFT stages
    int tap_bucket;  // taps rounded up to the compiled bucket
    int variant;     // bit 0: TMA ring; bit 1: twiddles in smem; bit 2: halo carried; bit 4: cluster
    const void* fn;  // kernel function (for occupancy queries and attributes)
    cudaError_t (*launch)(const FwdArgs&, int grid, cudaStream_t);
    int cluster;     // CTAs per thread-block cluster (0: none); grid counts CTAs
};

// Resident clusters of a cluster kernel entry (persistent grid): the most
// whole clusters of e.cluster CTAs that fit at once (0: none fits).
cudaError_t max_active_clusters(const FwdEntry& e, int sms, int* clusters);

struct BwdEntry {
    int threads;     // threads per CTA
    int batch;       // raw rows per CTA batch
    int smem;        // dynamic shared memory bytes
    const void* fn;
    cudaError_t (*launch)(const BwdArgs&, int grid, cudaStream_t);
};
// Adjoint kernels; false when (C, tap bucket, input type) is not built.
bool bwd_lookup(int C, int tap_bucket, int in, BwdEntry* e);
// grad_h[t*C + c] = sum_p partials[p*TM*C + t*C + c], p in order (NaN when *err != 0).
cudaError_t bwd_reduce(const float* partials, int nparts, int T, int TM, int C, const int* err, float* grad_h,
                       cudaStream_t st);

// Unfused adjoint (any planned shape): inverse DFT per C, then the
// transposed FIR and the tap correlation (runtime C and T).
struct IdftEntry {
    int threads;     // threads per CTA
    int batch;       // spectra per CTA batch
    int smem;        // dynamic shared memory bytes
    const void* fn;
    cudaError_t (*launch)(const IdftArgs&, int grid, cudaStream_t);
};
// grad_x pass; grid_x: CTAs along the row tiles of all streams.
cudaError_t bwd_gradx(const AdjFirArgs& a, int grid_x, cudaStream_t st);
// grad_h partial sums (a.n_parts parts of the rows of all streams).
cudaError_t bwd_gradh(int in, const AdjCorrArgs& a, cudaStream_t st);
// Tap blocks of the grad_h pass (partial-sum rows are TM*C floats).
int bwd_gradh_tap_blocks(int T);

// Per-C lookups; return false when the (tap bucket, in, out) triple is not built.
#define PPF_DECLARE_C(C)                                                         \
    bool fwd_lookup_c##C(int tap_bucket, int in, int out, FwdEntry* e);         \
    bool fir_lookup_c##C(int tap_bucket, int in, FwdEntry* e);                  \
    bool idft_lookup_c##C(IdftEntry* e);                                         \
    int fwd_twiddle_count_c##C();                                                \
    void fwd_twiddles_c##C(float* host_pairs);
PPF_DECLARE_C(32)
PPF_DECLARE_C(64)
PPF_DECLARE_C(128)
PPF_DECLARE_C(256)
PPF_DECLARE_C(512)
PPF_DECLARE_C(1024)
PPF_DECLARE_C(2048)
PPF_DECLARE_C(4096)
PPF_DECLARE_C(384)
PPF_DECLARE_C(768)
PPF_DECLARE_C(1536)
PPF_DECLARE_C(3072)
#undef PPF_DECLARE_C

}  // namespace ppf
