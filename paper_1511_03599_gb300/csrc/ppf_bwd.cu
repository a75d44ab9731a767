// ppf_bwd.cu -- instantiates the PFB adjoint kernels (complex FP32 input,
// C in {64, 128, 256}, tap buckets up to 16) and exports their lookup.
#include "ppf_bwd.cuh"
#include "ppf_internal.h"

namespace ppf {

template <int C, int TM>
static bool make_bwd(BwdEntry* e) {
    const BwdInfo i = bwd_info<C, TM>();
    if (i.fn == nullptr) return false;
    *e = BwdEntry{i.threads, i.batch, i.smem, i.fn, &bwd_launch<C, TM>};
    return true;
}

template <int C>
static bool bwd_by_tm(int tm, BwdEntry* e) {
    switch (tm) {
        case 1: return make_bwd<C, 1>(e);
        case 2: return make_bwd<C, 2>(e);
        case 4: return make_bwd<C, 4>(e);
        case 8: return make_bwd<C, 8>(e);
        case 16: return make_bwd<C, 16>(e);
        default: return false;
    }
}

bool bwd_lookup(int C, int tm, BwdEntry* e) {
    switch (C) {
        case 64: return bwd_by_tm<64>(tm, e);
        case 128: return bwd_by_tm<128>(tm, e);
        case 256: return bwd_by_tm<256>(tm, e);
        default: return false;
    }
}

cudaError_t bwd_reduce(const float* partials, int nparts, int T, int TM, int C, const int* err, float* grad_h,
                       cudaStream_t st) {
    const int TC = T * C;
    pfb_bwd_reduce_kernel<<<(TC + 255) / 256, 256, 0, st>>>(partials, nparts, TC, TM * C, err, grad_h);
    return cudaPeekAtLastError();
}

}  // namespace ppf
