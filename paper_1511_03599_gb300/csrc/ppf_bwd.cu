// ppf_bwd.cu -- instantiates the fused PFB adjoint kernels (complex int8 /
// int16 / FP32 input, C in {64, 128, 256, 512}, tap buckets up to 16 where
// the batch holds the halo) and the runtime-shape passes of the unfused
// adjoint, and exports their lookups and launches.
#include "ppf_bwd.cuh"
#include "ppf_bwd_unfused.cuh"
#include "ppf_internal.h"

namespace ppf {

template <int C, int TM, int IN>
static bool make_bwd(BwdEntry* e) {
    const BwdInfo i = bwd_info<C, TM, IN>();
    if (i.fn == nullptr) return false;
    *e = BwdEntry{i.threads, i.batch, i.smem, i.fn, &bwd_launch<C, TM, IN>};
    return true;
}

template <int C, int IN>
static bool bwd_by_tm(int tm, BwdEntry* e) {
    switch (tm) {
        case 1: return make_bwd<C, 1, IN>(e);
        case 2: return make_bwd<C, 2, IN>(e);
        case 4: return make_bwd<C, 4, IN>(e);
        case 8: return make_bwd<C, 8, IN>(e);
        case 16: return make_bwd<C, 16, IN>(e);
        default: return false;
    }
}

template <int C>
static bool bwd_by_in(int tm, int in, BwdEntry* e) {
    switch (in) {
        case IN_CI8: return bwd_by_tm<C, IN_CI8>(tm, e);
        case IN_CI16: return bwd_by_tm<C, IN_CI16>(tm, e);
        case IN_CF32: return bwd_by_tm<C, IN_CF32>(tm, e);
        default: return false;
    }
}

bool bwd_lookup(int C, int tm, int in, BwdEntry* e) {
    switch (C) {
        case 64: return bwd_by_in<64>(tm, in, e);
        case 128: return bwd_by_in<128>(tm, in, e);
        case 256: return bwd_by_in<256>(tm, in, e);
        case 512: return bwd_by_in<512>(tm, in, e);
        default: return false;
    }
}

cudaError_t bwd_reduce(const float* partials, int nparts, int T, int TM, int C, const int* err, float* grad_h,
                       cudaStream_t st) {
    const int TC = T * C;
    pfb_bwd_reduce_kernel<<<(TC + 255) / 256, 256, 0, st>>>(partials, nparts, TC, TM * C, err, grad_h);
    return cudaPeekAtLastError();
}

cudaError_t bwd_gradx(const AdjFirArgs& a, int grid_x, cudaStream_t st) {
    const int pairs = a.C / 2, nt = pairs < 128 ? pairs : 128;
    pfb_bwd_gradx_kernel<<<dim3(grid_x, (pairs + nt - 1) / nt), nt, 0, st>>>(a);
    return cudaPeekAtLastError();
}

int bwd_gradh_tap_blocks(int T) { return (T + kAdjTB - 1) / kAdjTB; }

cudaError_t bwd_gradh(int in, const AdjCorrArgs& a, cudaStream_t st) {
    const int pairs = a.C / 2, nt = pairs < 128 ? pairs : 128;
    const dim3 grid(a.n_parts, (pairs + nt - 1) / nt, bwd_gradh_tap_blocks(a.T));
    switch (in) {
        case IN_CI8: pfb_bwd_gradh_kernel<IN_CI8><<<grid, nt, 0, st>>>(a); break;
        case IN_CI16: pfb_bwd_gradh_kernel<IN_CI16><<<grid, nt, 0, st>>>(a); break;
        case IN_CF32: pfb_bwd_gradh_kernel<IN_CF32><<<grid, nt, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaPeekAtLastError();
}

}  // namespace ppf
