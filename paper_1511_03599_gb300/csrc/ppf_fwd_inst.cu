// ppf_fwd_inst.cu -- instantiates the fused forward kernel for one channel
// count C (compiled once per C with -DPPF_C=<C>) over every tap bucket,
// input type and output type, and the inverse DFT of the unfused adjoint,
// and exports the lookups used by the C ABI.
#include "ppf_bwd_unfused.cuh"
#include "ppf_fwd.cuh"
#include "ppf_internal.h"

#ifndef PPF_C
#error "compile with -DPPF_C=<channels>"
#endif

#define PPF_CAT2(a, b) a##b
#define PPF_CAT(a, b) PPF_CAT2(a, b)

namespace ppf {

template <int TM, int IN, int OUT>
static bool make_entry(FwdEntry* e) {
    FwdInfo i = fwd_info<PPF_C, TM, IN, OUT>();
    *e = FwdEntry{i.threads, i.batch, i.smem, i.stages, i.tap_bucket, i.variant, i.fn, &fwd_launch<PPF_C, TM, IN, OUT>,
                  i.cluster};
    return true;
}

template <int TM, int IN>
static bool by_out(int out, FwdEntry* e) {
    switch (out) {
        case OUT_CF32: return make_entry<TM, IN, OUT_CF32>(e);
        case OUT_CF16: return make_entry<TM, IN, OUT_CF16>(e);
        default: return false;
    }
}

template <int TM>
static bool by_in(int in, int out, FwdEntry* e) {
    switch (in) {
        case IN_CI8: return by_out<TM, IN_CI8>(out, e);
        case IN_CI16: return by_out<TM, IN_CI16>(out, e);
        case IN_CF32: return by_out<TM, IN_CF32>(out, e);
        default: return false;
    }
}

bool PPF_CAT(fwd_lookup_c, PPF_C)(int tm, int in, int out, FwdEntry* e) {
    switch (tm) {
        case 1: return by_in<1>(in, out, e);
        case 2: return by_in<2>(in, out, e);
        case 4: return by_in<4>(in, out, e);
        case 8: return by_in<8>(in, out, e);
        case 16: return by_in<16>(in, out, e);
        case 64: return by_in<64>(in, out, e);   // any T in 17..64 (runtime tap loop)
        default: return false;
    }
}

template <int TM, int IN>
static bool make_fir(FwdEntry* e) {
    FwdInfo i;
    if (!fir_info<PPF_C, TM, IN>(&i)) return false;
    *e = FwdEntry{i.threads, i.batch, i.smem, i.stages, i.tap_bucket, i.variant, i.fn, &fir_launch<PPF_C, TM, IN>, 0};
    return true;
}

template <int TM>
static bool fir_by_in(int in, FwdEntry* e) {
    switch (in) {
        case IN_CI8: return make_fir<TM, IN_CI8>(e);
        case IN_CI16: return make_fir<TM, IN_CI16>(e);
        case IN_CF32: return make_fir<TM, IN_CF32>(e);
        default: return false;
    }
}

bool PPF_CAT(fir_lookup_c, PPF_C)(int tm, int in, FwdEntry* e) {
    switch (tm) {
        case 1: return fir_by_in<1>(in, e);
        case 2: return fir_by_in<2>(in, e);
        case 4: return fir_by_in<4>(in, e);
        case 8: return fir_by_in<8>(in, e);
        case 16: return fir_by_in<16>(in, e);
        default: return false;
    }
}

bool PPF_CAT(idft_lookup_c, PPF_C)(IdftEntry* e) {
    const IdftInfo i = idft_info<PPF_C>();
    *e = IdftEntry{i.threads, i.batch, i.smem, i.fn, &idft_launch<PPF_C>};
    return true;
}

int PPF_CAT(fwd_twiddle_count_c, PPF_C)() { return tw_total_float2s(PPF_C) > 0 ? tw_total_float2s(PPF_C) : 1; }

void PPF_CAT(fwd_twiddles_c, PPF_C)(float* host_pairs) {
    fill_twiddles<PPF_C>(reinterpret_cast<float2*>(host_pairs));
}

}  // namespace ppf
