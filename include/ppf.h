/*
 * ppf.h -- C ABI of the GB300 polyphase filter bank (PFB) channeliser.
 *
 * Method: Adamek, Novotny & Armour, "A polyphase filter for many-core
 * architectures" (arXiv:1511.03599).  For a complex stream split into raw
 * spectra of C channels ("contiguous in channels", Sec. 3.1) the PFB is
 *
 *   FIR (Alg. 1, Sec. 3.2):
 *     y[s][c] = sum_{t=0}^{T-1} h[t*C + c] * x[(s+t)*C + c]
 *   DFT (Eq. 2, Sec. 2), unnormalised, sign -i, natural bin order:
 *     Y[s][m] = sum_{c=0}^{C-1} y[s][c] * exp(-2 pi i c m / C)
 *
 * for output spectra s = 0 .. n_spectra-1.  Output spectrum s reads raw
 * spectra s .. s+T-1, so the input holds C*(n_spectra+T-1) samples and there
 * is no zero-padded history.  Eq. 1 as printed has a garbled index; this
 * library follows the index convention of Alg. 1-3 (oldest raw spectrum
 * paired with tap block 0).  A caller wanting the convolution convention
 * reverses the tap blocks on the host.
 *
 * Both steps run in one CUDA kernel on one GPU (sm_103a); the filtered
 * spectra y never leave the SM.  Accumulation is FP32 throughout.
 *
 * Conventions of every entry point:
 *   - status codes only: nothing throws, exits or traps;
 *   - device pointers are caller-owned, must be 16-byte aligned and must not
 *     overlap; host pointers are read during the call only;
 *   - work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising, except where noted;
 *   - a plan is bound to the device that was current when it was made.
 */
#ifndef PPF_H
#define PPF_H

#ifdef __cplusplus
extern "C" {
#endif

/* Input sample types: complex, interleaved (re, im) (Sec. 3.1 input precisions).
 * Integers are two's complement; the value is the integer, no offset or scale. */
typedef enum {
    PPF_IN_CI8 = 0,   /* 2 bytes per sample: int8 re, int8 im   */
    PPF_IN_CI16 = 1,  /* 4 bytes per sample: int16 re, int16 im */
    PPF_IN_CF32 = 2   /* 8 bytes per sample: float re, float im */
} ppf_in_t;

/* Output sample types: complex FP32 (8 bytes) or complex FP16 (4 bytes,
 * interleaved half re, half im; round-to-nearest-even from the FP32 result,
 * +-inf on overflow).  The paper always writes 32-bit outputs (Sec. 3.1);
 * FP16 is an extension. */
typedef enum {
    PPF_OUT_CF32 = 0,
    PPF_OUT_CF16 = 1
} ppf_out_t;

typedef enum {
    PPF_OK = 0,
    PPF_ERR_INVALID_ARG = 1,     /* null pointer, C<1, T<1, n_spectra<1, overlap, bad handle */
    PPF_ERR_UNSUPPORTED = 2,     /* C not supported (see ppf_plan), T > 64, unknown dtype */
    PPF_ERR_ALIGNMENT = 3,       /* a buffer is not 16-byte aligned */
    PPF_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed */
    PPF_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side wait gave up (see ppf_device_status) */
    PPF_ERR_OUT_OF_MEMORY = 6    /* a device or pinned-host allocation failed */
} ppf_status;

typedef struct ppf_plan_s* ppf_plan_t;
typedef struct ppf_beams_s* ppf_beams_t;
typedef void* ppf_stream_t;     /* cudaStream_t */

/* Largest supported values. */
#define PPF_MIN_CHANNELS 32
#define PPF_MAX_CHANNELS 4096
#define PPF_MAX_TAPS 64

/*
 * ppf_plan -- validate (C, T, types), copy the C*T FP32 coefficients to
 * device memory owned by the plan and pick the kernel for the shapes.
 *   out        : receives the plan handle (set to NULL on failure)
 *   C          : channels per spectrum: a power of two in [32, 4096], or
 *                3*2^k in {384, 768, 1536, 3072} (mixed-radix DFT with a
 *                radix-3 stage; the paper's non-power-of-two example is
 *                C = 3072, Sec. 4.2 / 5.3).  The paper needs C divisible by 32
 *                (Sec. 4.1).
 *   T          : taps, 1 <= T <= 64
 *   coeffs_host: C*T host floats, tap-major: coeffs_host[t*C + c] is tap t of
 *                channel c (coefficients are unique per channel and tap and
 *                always FP32, Sec. 3.1).  Read during the call only.
 * Allocates device memory (cudaMalloc); synchronous.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, OUT_OF_MEMORY.
 */
ppf_status ppf_plan(ppf_plan_t* out, int C, int T, const float* coeffs_host,
                    ppf_in_t in_dtype, ppf_out_t out_dtype);

/*
 * ppf_execute -- enqueue the fused FIR + DFT on `stream`.
 *   in_dev   : device buffer of C*(n_spectra+T-1) input samples (in_dtype)
 *   out_dev  : device buffer of n_spectra*C output samples (out_dtype),
 *              spectrum-major: out[s*C + m] = Y[s][m]
 *   n_spectra: output spectra, >= 1
 * A long stream is processed in chunks that overlap by T-1 raw spectra.
 * Asynchronous; one kernel launch; no allocation.
 * Errors: INVALID_ARG, ALIGNMENT, CUDA (launch failure).
 */
ppf_status ppf_execute(ppf_plan_t plan, const void* in_dev, void* out_dev,
                       long long n_spectra, ppf_stream_t stream);

/*
 * ppf_execute_batched -- ppf_execute over n_streams independent streams (beams)
 * in one launch.  Stream i reads in_dev + i*in_stride samples and writes
 * out_dev + i*out_stride samples; strides are in samples (elements of
 * in_dtype / out_dtype pairs), at least one stream long, and their byte
 * sizes multiples of 16.  CTAs are spread over the streams; each stream is
 * transformed exactly as ppf_execute would.  Asynchronous; one launch.
 * Errors: INVALID_ARG, ALIGNMENT, CUDA.
 */
ppf_status ppf_execute_batched(ppf_plan_t plan, const void* in_dev, long long in_stride, void* out_dev,
                               long long out_stride, long long n_spectra, long long n_streams,
                               ppf_stream_t stream);

/*
 * ppf_backward -- adjoint of the transform, for fitting the taps by gradient
 * descent.  Conjugate-Wirtinger convention (PyTorch's): for a real loss L and
 * complex z the gradient is dL/dRe(z) + i dL/dIm(z).  With G = grad_out:
 *   g_y = F^H G (unnormalised inverse DFT, sign +i, per spectrum),
 *   grad_in[r][c]   = sum_t h[t*C+c] g_y[r-t][c],
 *   grad_taps[t*C+c] = sum over streams and s of Re(conj(g_y[s][c]) x[s+t][c]).
 *   grad_out_dev : n_streams * n_spectra*C complex FP32, streams contiguous
 *   in_dev       : the forward input, n_streams * C*(n_spectra+T-1) samples of
 *                  the plan's input type (complex int8 / int16 / FP32)
 *   grad_in_dev  : n_streams * C*(n_spectra+T-1) complex FP32, one per input
 *                  sample (written, not accumulated), or NULL
 *   grad_taps_dev: C*T floats (written), or NULL; not both NULL
 * Every shape the plan accepts is supported.  For C in [64, 512] with
 * T <= 16 (T <= 8 at C = 512) one fused kernel computes all three sums; for
 * the other shapes (C = 32, C >= 1024, C = 3*2^k, T = 17..64, and T > 8 at
 * C = 512) three passes run instead: the inverse DFT into a g_y scratch of
 * n_streams*n_spectra*C complex FP32 owned by the plan, then grad_in, then
 * the tap-gradient partial sums.  grad_in must not overlap grad_out or the
 * input.  The tap gradient is a deterministic two-pass reduction (partial
 * sums per CTA or per part of the rows, then a fixed-order sum).  The
 * partial-sum and g_y scratch are allocated by the plan on the first call
 * and grown when a call needs more (cudaMalloc inside the call).
 * Asynchronous on `stream`.
 * If a bounded device wait gives up (ppf_check_device then reports
 * PPF_ERR_DEVICE_TIMEOUT), grad_in is incomplete and every element of
 * grad_taps is NaN; the plan's status word stays set until ppf_check_device
 * clears it, and tap gradients computed meanwhile are NaN too.
 * Errors: INVALID_ARG, UNSUPPORTED, ALIGNMENT, CUDA, OUT_OF_MEMORY.
 */
ppf_status ppf_backward(ppf_plan_t plan, const void* grad_out_dev, const void* in_dev, void* grad_in_dev,
                        float* grad_taps_dev, long long n_spectra, long long n_streams, ppf_stream_t stream);

/*
 * ppf_backward_noalloc -- ppf_backward for callers that cannot allocate device
 * memory where they run it (a processing loop with a device-memory budget
 * fixed at start-up, or code where a cudaMalloc -- which may synchronise the
 * device or fail under memory pressure -- is not allowed).  The paper has no
 * counterpart; this is a deployment convenience.  Same arguments, results
 * and errors as ppf_backward for the shapes of its fused kernel (C in
 * [64, 512], T <= 16, T <= 8 at C = 512; other shapes: UNSUPPORTED, since the
 * three-pass path needs a g_y scratch), but the per-CTA tap-gradient partial
 * sums live in one fixed 2 MiB array (524,288 floats) inside the library
 * instead of plan memory, and the call allocates nothing.  The plan itself (made once
 * at set-up with ppf_plan) still owns the taps and tables.
 *   - Size limit: each CTA needs a row of tap_bucket*C floats; the call uses
 *     at most 524,288 / (tap_bucket*C) CTAs (128 at C=256, T=16 or C=512,
 *     T=8, fewer than the GPU holds at once there).  CTAs share the batches
 *     of all streams, so every stream count fits.
 *   - The first call on a device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress); make that first call before
 *     any stream capture.
 *   - Every call on a device shares that device's array, which keeps the last
 *     call's contents; each call overwrites all the rows it reads, so nothing
 *     needs clearing.  Calls on one device that overlap on the GPU (for
 *     instance on two streams) race on the array: order them.
 *   - Every GPU that loads the library holds the array until process exit.
 */
ppf_status ppf_backward_noalloc(ppf_plan_t plan, const void* grad_out_dev, const void* in_dev, void* grad_in_dev,
                                float* grad_taps_dev, long long n_spectra, long long n_streams,
                                ppf_stream_t stream);

/*
 * ppf_update_taps -- replace the plan's C*T coefficients (tap-major, FP32)
 * with those at taps_dev (device memory), ordered on `stream`: launches
 * enqueued after it use the new taps.  Used when fitting the taps.
 * Asynchronous; no allocation.  Errors: INVALID_ARG, CUDA.
 */
ppf_status ppf_update_taps(ppf_plan_t plan, const float* taps_dev, ppf_stream_t stream);

/*
 * Multi-beam channelisation in one persistent launch (many independent beams
 * with uneven C, T and spectrum counts, e.g. the sub-bands of a receiver).
 *
 * ppf_beams_plan -- n_beams beams; beam i has C[i] channels (a power of two
 *   in [64, 4096]), T[i] <= 16 taps, n_spectra[i] output spectra and taps_host[i]
 *   (C[i]*T[i] FP32, tap-major; read during the call).  Complex int8 input and
 *   complex FP32 output only (else UNSUPPORTED).  The plan cuts every beam
 *   into tiles of about 2^20 samples, sorts them largest first into a wide
 *   (C >= 1024) and a narrow queue and keeps taps, twiddles, descriptors,
 *   tiles, two work-queue counters and a status word in device memory it
 *   allocates.  Synchronous.
 * ppf_beams_bind -- the device buffers of every beam (in_dev[i]: C[i]*(n_spectra[i]
 *   +T[i]-1) samples, out_dev[i]: n_spectra[i]*C[i] outputs; 16-byte aligned);
 *   copied to the device descriptors (synchronous).  Rebind when they change.
 * ppf_beams_set_tiling -- re-cut the tiles to about tile_samples samples each
 *   (the autotuner's knob); synchronous.
 * ppf_beams_execute -- enqueue one reset of the two queue counters and ONE
 *   launch of the persistent kernel (one CTA of 512 threads per SM;
 *   ctas_per_sm is accepted for compatibility and clamped to what fits).
 *   Each CTA first pulls wide tiles (beams with C >= 1024) and runs each with
 *   all its threads, then splits into two groups of 256 threads that pull
 *   narrow tiles (C <= 512) independently.  A tile runs the FIR + DFT body of
 *   a single-stream kernel: the carry kernel's at C = 1024 (FIR halo carried
 *   in registers), the generic kernel's otherwise (raw rows staged through a
 *   TMA ring).  Every beam's result equals ppf_execute's up to FP32 rounding
 *   (bit-identical at C = 1024 with up to 8 taps and at C = 4096, where
 *   ppf_execute runs the same body).  Asynchronous on `stream`; no allocation.
 * ppf_beams_info -- info[0]=beams, [1]=tiles, [2]=tile samples, [3]=CTAs per SM,
 *   [4]=SMs, [5]=dynamic shared memory bytes, [6]=wide tiles (C >= 1024).
 * ppf_beams_check_device -- as ppf_check_device, for the multi-beam launch.
 * ppf_beams_destroy -- free everything (NULL accepted).
 * Errors: INVALID_ARG, UNSUPPORTED, ALIGNMENT, CUDA, OUT_OF_MEMORY, DEVICE_TIMEOUT.
 */
ppf_status ppf_beams_plan(ppf_beams_t* out, int n_beams, const int* C, const int* T, const long long* n_spectra,
                          const float* const* taps_host, ppf_in_t in_dtype, ppf_out_t out_dtype);
ppf_status ppf_beams_bind(ppf_beams_t beams, const void* const* in_dev, void* const* out_dev);
ppf_status ppf_beams_set_tiling(ppf_beams_t beams, long long tile_samples);
ppf_status ppf_beams_execute(ppf_beams_t beams, int ctas_per_sm, ppf_stream_t stream);
ppf_status ppf_beams_info(ppf_beams_t beams, long long info[7]);
ppf_status ppf_beams_check_device(ppf_beams_t beams, ppf_stream_t stream);
ppf_status ppf_beams_destroy(ppf_beams_t beams);

/*
 * ppf_fir / ppf_fft -- the unfused form of the same transform, for the
 * ablation that measures what fusion saves (the paper runs a FIR kernel and
 * then a batched FFT library call, Sec. 3.2).
 *   ppf_fir: the FIR alone (Alg. 1): in_dev as for ppf_execute, y_dev
 *            receives n_spectra*C complex FP32 filtered samples y[s][c].
 *            Exists where the carry kernel's FIR fits (halo in registers):
 *            C in {64, 128, 256, 512} (and 1024 for int8 input), T <= 16
 *            (else UNSUPPORTED); at C = 1024 with 9-16 taps the fused path
 *            itself runs the generic kernel.
 *   ppf_fft: the DFT alone (Eq. 2) of n_spectra rows of C complex FP32 values
 *            at y_dev into out_dev (the plan's output type); runs the fused
 *            kernel with T = 1 and unit taps (exact); its internal plan is
 *            made on the first call (allocates a few KB).
 * ppf_fft(ppf_fir(x)) equals ppf_execute(x) up to FP32 rounding.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, UNSUPPORTED, ALIGNMENT, CUDA.
 */
ppf_status ppf_fir(ppf_plan_t plan, const void* in_dev, void* y_dev, long long n_spectra, ppf_stream_t stream);
ppf_status ppf_fft(ppf_plan_t plan, const void* y_dev, void* out_dev, long long n_spectra, ppf_stream_t stream);

/*
 * ppf_execute_host -- the same transform with HOST input and output buffers.
 * The stream is cut into chunks (about 64 MiB of output each) that are
 * copied host->device, transformed and copied device->host on three CUDA
 * streams, one per engine, so that the copies of chunk i+1 and i-1 overlap
 * the compute of chunk i (the copy / compute overlap of Sec. 5) with at most
 * one copy per direction in flight.  Three device staging slots per
 * direction are allocated on the first call and kept by the plan.  Pinned host buffers give full copy speed;
 * pageable ones work but are slower.  Synchronous: returns when `out_host`
 * holds the result.  `stream` orders the call after earlier work on it.
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY.
 */
ppf_status ppf_execute_host(ppf_plan_t plan, const void* in_host, void* out_host,
                            long long n_spectra, ppf_stream_t stream);

/* ppf_destroy -- free the plan and its device memory (synchronises the device
 * work of the plan's own streams).  NULL is accepted. */
ppf_status ppf_destroy(ppf_plan_t plan);

/* Human-readable name of a status code (static string). */
const char* ppf_status_string(ppf_status s);

/* Detail of the last error raised on the calling thread (static buffer). */
const char* ppf_last_error_message(void);

/* Plan introspection: launch shape chosen for the plan.
 *   info[0]=threads per CTA, info[1]=spectra per CTA batch, info[2]=grid
 *   (CTAs), info[3]=dynamic shared memory bytes, info[4]=tap bucket (T
 *   rounded up), info[5]=number of FFT stages, info[6]=kernel variant
 *   (bit 0: raw input staged through a TMA ring in shared memory; bit 1:
 *   twiddles in shared memory; bit 2: FIR halo carried in registers between
 *   batches; bit 4: thread-block-cluster kernel, info[2] then counts the
 *   CTAs of whole clusters; bit 5: the cluster's CTAs push their filtered
 *   channels into the transforming CTA's shared memory; bit 6: long-tap
 *   kernel, T = 17..64, raw rows and halo streamed through a TMA ring),
 *   info[7]=CTAs resident per SM. */
ppf_status ppf_plan_info(ppf_plan_t plan, int info[8]);

/*
 * ppf_check_device -- read (and clear) the plan's device status word after
 * the work queued on `stream`.  Every device-side wait of the kernels is
 * bounded; one that gives up makes its CTA return early and sets the word.
 * Synchronises `stream`.  Returns PPF_OK or PPF_ERR_DEVICE_TIMEOUT (the
 * outputs of the affected launch are then incomplete); the context stays
 * usable.  Errors: INVALID_ARG, CUDA.
 */
ppf_status ppf_check_device(ppf_plan_t plan, ppf_stream_t stream);

/*
 * ppf_set_debug_flags -- testing aids, a bitwise OR of:
 *   PPF_DEBUG_INJECT_TIMEOUT (1): every later launch of the plan's
 *     staged-input kernel waits on a barrier that nothing completes, so the
 *     bounded wait runs out (after 2 ms) and the timeout path is exercised
 *     without faulting the GPU;
 *   PPF_DEBUG_UNFUSED_ADJOINT (2): ppf_backward runs its three-pass path even
 *     where the fused adjoint kernel exists (to compare the two paths;
 *     ppf_backward_noalloc ignores it).
 * flags = 0 restores normal operation.  Errors: INVALID_ARG (unknown bit).
 */
#define PPF_DEBUG_INJECT_TIMEOUT 1
#define PPF_DEBUG_UNFUSED_ADJOINT 2
ppf_status ppf_set_debug_flags(ppf_plan_t plan, int flags);

/*
 * ppf_probe_rates -- throughput micro-benchmarks of the current device, the
 * analogue of the paper's type-conversion and bandwidth micro-benchmarks
 * (Sec. 4.1, Table 3).  Writes up to n rates, in operations per second:
 *   [0] scalar FP32 FMA, [1] packed f32x2 FMA (two per instruction),
 *   [2] int8 -> FP32 conversions (compiler conversion instruction),
 *   [3] int8 -> FP32 conversions by exponent-bias byte placement,
 *   [4] int16 -> FP32 conversions.
 * Synchronous (legacy default stream); allocates a small device buffer.
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY.
 */
ppf_status ppf_probe_rates(double* rates, int n);

/*
 * ppf_probe_stream -- achievable DRAM bandwidth for a traffic mix: a streaming
 * kernel reads in_bytes from in_dev and writes ratio*in_bytes to out_dev
 * (16-byte vectors, coalesced, streaming hints); *bytes_per_s receives
 * (1+ratio)*in_bytes / time (best of three timings of three launches,
 * after a warm-up launch).  The PFB
 * with int8 input and complex FP32 output moves 1 byte in per 4 out.
 * Buffers are caller-owned device memory, 16-byte aligned, in_bytes a
 * multiple of 16, 0 <= ratio <= 16.  Synchronous (legacy default stream).
 * Errors: INVALID_ARG, CUDA.
 */
ppf_status ppf_probe_stream(const void* in_dev, void* out_dev, long long in_bytes, int ratio, double* bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* PPF_H */
