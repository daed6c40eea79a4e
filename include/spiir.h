/*
 * spiir.h -- C ABI of the SPIIR filter-bank library for NVIDIA B300 (sm_103a).
 *
 * The operation (paper, section "GPU accelerated SPIIR method", subsection
 * "SPIIR method"): every template of a bank is approximated by a parallel
 * bank of single-pole complex IIR filters,
 *
 *     y_l[k] = a_l * y_l[k-1] + b_l * x[k - d_l],      z[k] = sum_l y_l[k],
 *
 * run on whitened detector strain x; z is the template's complex SNR series
 * and its peak (largest |z|) flags a candidate signal.  The per-template
 * parameter triples (a_l, b_l, d_l) are the "parameter array" of subsection
 * "Optimized GPU implementation of SPIIR", which this library repacks into an
 * aligned, coalesced device layout when a plan is created.
 *
 * Conventions shared by every call:
 *  - Complex numbers are interleaved (re, im) float32 pairs (complex64).
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers without the suffix are host memory,
 *    read (or written) only during the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued asynchronously on it; a call returning
 *    SPIIR_OK means the work was enqueued, not that it finished.
 *  - No call aborts, exits or throws.  Every failure returns a status and
 *    records a one-line reason readable with spiir_last_error_detail()
 *    (per host thread).
 *  - A plan is not thread-safe; distinct plans may be used from distinct host
 *    threads.  All calls on one plan must use streams ordered with each other
 *    (the plan owns the filter state and the strain history).
 *  - There is no CPU fallback: without a B300-class device the compute calls
 *    return SPIIR_EUNSUPPORTED or SPIIR_ECUDA.
 */
#ifndef SPIIR_H
#define SPIIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spiir_status {
    SPIIR_OK = 0,
    SPIIR_EINVAL = 1,       /* bad argument: null pointer, size, |a| >= 1, d < 0 ... */
    SPIIR_ENOMEM = 2,       /* host or device allocation failed                     */
    SPIIR_ECUDA = 3,        /* a CUDA runtime call failed                           */
    SPIIR_ETIMEOUT = 4,     /* a bounded device-side wait gave up (error word set)  */
    SPIIR_EUNSUPPORTED = 5  /* device is not sm_103, or a size beyond a kernel limit */
} spiir_status;

/* How the recurrence is evaluated (see spiir_options.precision). */
typedef enum spiir_precision {
    SPIIR_PREC_PLAIN = 0,       /* complex FP32 state, one pass over time          */
    SPIIR_PREC_COMPENSATED = 1, /* float-float (two-sum/two-prod) state            */
    SPIIR_PREC_CHUNKED_FP64 = 2,/* time-chunked scan, FP64 carry of the state      */
    SPIIR_PREC_CHUNKED_TC = 3   /* chunked scan, split-BF16 tensor-core projection */
} spiir_precision;

/* Segment start states of time-segmented calls (spiir_options.projection). */
typedef enum spiir_projection {
    SPIIR_PROJECT_AUTO = 0,
    SPIIR_PROJECT_RECURRENCE = 1,
    SPIIR_PROJECT_TENSOR = 2
} spiir_projection;

/*
 * A template bank in CSR form.  Template t owns filters
 * filter_off[t] .. filter_off[t+1]-1.  All arrays are host memory, read only
 * during spiir_plan_create; the plan copies what it needs.
 *   n_templates      >= 1
 *   n_detectors      >= 1; every template is run on every detector stream
 *   filter_off       [n_templates + 1], filter_off[0] = 0, non-decreasing
 *   a_reim, b_reim   [2 * Ltot] complex64 pole and gain; |a_l| < 1 required
 *   delay            [Ltot] delay d_l >= 0, in samples of the filter's band
 *   n_bands          0 (or 1 with band_decim[0] = 1): single-rate bank.
 *                    > 1: multirate bank (see spiir_filter)
 *   band_of_filter   [Ltot] band index of each filter, or NULL if n_bands <= 1
 *   band_decim       [n_bands] decimation factor of each band relative to the
 *                    top rate (1 = top rate), or NULL if n_bands <= 1
 */
typedef struct spiir_bank_desc {
    int64_t n_templates;
    int32_t n_detectors;
    int32_t n_bands;
    const int64_t *filter_off;
    const float *a_reim;
    const float *b_reim;
    const int32_t *delay;
    const int32_t *band_of_filter;
    const int32_t *band_decim;
} spiir_bank_desc;

/* Plan options.  Fill with spiir_options_default() and override fields. */
typedef struct spiir_options {
    int32_t precision;      /* spiir_precision                                   */
    int32_t chunk_len;      /* chunked forms: samples per chunk (default 256)     */
    int32_t block_len;      /* samples per staged strain block; 0 = default       */
    int32_t warps_per_cta;  /* templates per CTA; 0 = chosen from the bank size   */
    int32_t ring_copies;    /* bank-skewed copies of the strain ring: 1, 2 or 4;  */
                            /* 0 = default: 2 for full-warp layouts of at most 4  */
                            /* filters per lane (per band), else 1               */
    int32_t device;         /* CUDA device ordinal; -1 = host-only plan (layout    */
                            /* and statistics, no device memory, no compute)       */
    int32_t autotune;       /* nonzero: time candidate block/copy settings on the  */
                            /* first spiir_filter call and keep the fastest (a     */
                            /* bank whose calls run in time segments keeps the     */
                            /* default layout)                                     */
    int32_t max_filters_per_lane; /* 1..10 filters held per thread; templates with */
                            /* more than 32x this many filters span several warps; */
                            /* 0 = default (10)                                    */
    int32_t lanes_per_template; /* 32, or 16 (two templates per warp, for small     */
                            /* templates); 0 = 16 when every template has at most  */
                            /* 96 filters (and 16 x max_filters_per_lane) and the  */
                            /* bank still fills >= 16 warps per SM at 16 lanes     */
    int32_t time_segments;  /* plain precision: split each call into this many time */
                            /* segments run in parallel, each from its start state */
                            /* given by the projection below (segments are >= 1    */
                            /* block long; spiir_filter_backward splits its reverse */
                            /* pass into as many whole checkpoint intervals, auto: */
                            /* ~4 waves of 16 warps/SM).  0 = auto: banks that fill */
                            /* < 1/8                                               */
                            /* of the GPU's warps get up to 8 warps/SM worth (>= 4  */
                            /* segments, <= 64), banks under one full wave (16     */
                            /* warps/SM) get 2 on calls of >= 64 blocks, others    */
                            /* none; 1 = off.  Results of different splits agree   */
                            /* to rounding, not bit for bit                        */
    int32_t projection;     /* how segmented calls get their segment start states: */
                            /* SPIIR_PROJECT_AUTO (= TENSOR), _RECURRENCE (a zero-  */
                            /* state FP32 pass over all but the last segment, FP64 */
                            /* carry) or _TENSOR (chunk sums by split-BF16 tcgen05 */
                            /* GEMM, FP32 chunk scan)                              */
    int32_t kernel_timing;  /* nonzero: record CUDA events around every filter   */
                            /* (K1) and tensor-core projection launch, outside     */
                            /* stream capture; read them with spiir_kernel_times  */
    int32_t tile_chunks;    /* chunked_tc: 256-sample chunks per time tile (the    */
                            /* anchors of one tile are held at once); 0 = auto:    */
                            /* anchors within a quarter of free memory, <= 16 GiB */
    int32_t persistent;     /* unsegmented plain calls: 1 = one CTA per (CTA group,  */
                            /* detector) unit, in launch order largest first (the   */
                            /* hardware starts each CTA where one has finished);   */
                            /* 2 = persistent: as many CTAs as fit on the GPU at    */
                            /* once take the units, largest first, from a device    */
                            /* counter; 0 = auto: 1, or what the autotuner picked   */
    int32_t tail_split;     /* plain single-rate banks: the smallest templates run  */
                            /* on twice their warps so the launch ends on short     */
                            /* units.  0 = off, -1 = auto (the split, up to 20% of  */
                            /* the bank's filter rounds, with the shortest         */
                            /* predicted launch on the resident CTAs), k in 1..200 */
                            /* = the smallest templates holding k per mille of the  */
                            /* filter rounds                                        */
    int32_t adjoint_form;   /* how spiir_filter_backward evaluates g_a and g_b:     */
                            /* SPIIR_ADJOINT_REVERSE (the reverse-time recurrence   */
                            /* over a checkpointed forward), _TANGENT (one forward  */
                            /* pass of each filter's derivative recurrences, no     */
                            /* checkpoints) or _AUTO (tangent for calls of <= 8192  */
                            /* samples, and when the bank holds >= 8 warps per SM  */
                            /* at one filter per thread, >= 2 without grad_x)      */
    int32_t reserved[1];
} spiir_options;

/* Evaluation of the adjoint's g_a, g_b (spiir_options.adjoint_form). */
typedef enum spiir_adjoint_form {
    SPIIR_ADJOINT_AUTO = 0,
    SPIIR_ADJOINT_REVERSE = 1,
    SPIIR_ADJOINT_TANGENT = 2
} spiir_adjoint_form;

/* Plan statistics (spiir_plan_get_info). */
typedef struct spiir_plan_info {
    int64_t n_templates;
    int64_t n_filters;          /* Ltot                                          */
    int64_t n_slots;            /* filter slots incl. padding (per detector)      */
    int64_t n_units;            /* CTA work units per spiir_filter launch         */
    int32_t n_detectors;
    int32_t warps_per_cta;
    int32_t block_len;
    int32_t ring_copies;
    int32_t history_len;        /* strain samples kept between calls (>= max d)   */
    int32_t smem_bytes;         /* dynamic shared memory per CTA                  */
    int32_t max_filters_per_lane; /* largest filters per thread in any CTA        */
    int32_t precision;
    double bank_conflict_ratio; /* mean shared-memory wavefronts per strain load  */
    int32_t lanes_per_template; /* 32, or 16 when two templates share a warp        */
    int32_t last_call_launches; /* kernels the last spiir_filter or                 */
                                /* spiir_filter_backward call launched (not counting */
                                /* the autotuner's first-call timing launches)       */
    int32_t last_call_segments; /* time segments of the last spiir_filter call      */
    int32_t persistent;         /* 1: unsegmented plain calls launch persistent CTAs */
                                /* (the option, or the autotuner's choice)            */
    int64_t tail_templates;     /* templates the tail split gave twice their warps   */
    int64_t resident_ctas;      /* resident CTAs the tail split's launch model used  */
} spiir_plan_info;

typedef struct spiir_plan spiir_plan;

/* Fill *opt with defaults (plain precision, device 0). */
void spiir_options_default(spiir_options *opt);

/*
 * Validate the bank, sort templates by filter count, pack the parameter
 * array, and (device >= 0) allocate the plan's device state on that device
 * (subsection "Optimized GPU implementation of SPIIR": the per-template
 * parameter arrays are packed aligned and contiguous, and templates are
 * mapped to warps or blocks by their filter count).
 * Errors: EINVAL (bad bank or options), ENOMEM, ECUDA, EUNSUPPORTED (device
 * is not compute capability 10.3, or a template is beyond the kernels'
 * limits).  On error *out is set to NULL.
 */
spiir_status spiir_plan_create(const spiir_bank_desc *bank, const spiir_options *opt,
                               spiir_plan **out);

/* Free everything the plan owns (waits for its device work).  NULL is OK. */
spiir_status spiir_plan_destroy(spiir_plan *plan);

/* Statistics of the plan's layout.  Works for host-only plans. */
spiir_status spiir_plan_get_info(const spiir_plan *plan, spiir_plan_info *info);

/* The autotuner's timings, one "cap/W/C/Tb/tail=ms" entry per candidate
 * layout ("" before the first call of an autotuned plan, or without
 * autotune; "skipped: ..." when the first call ran in time segments).  The string belongs to the plan and lives until its next
 * spiir_filter call or its destruction. */
const char *spiir_plan_tune_report(const spiir_plan *plan);

/*
 * Slot map of a plan, for inspection: slot_filter[s] is the bank filter index
 * packed in slot s, or -1 for padding; slot_template[s] the template it
 * serves (-1 for an empty warp).  Both arrays are host memory of
 * info.n_slots entries (for multirate banks: the slots of every band, band
 * after band).
 */
spiir_status spiir_plan_get_slots(const spiir_plan *plan, int64_t *slot_filter,
                                  int64_t *slot_template);

/* Zero the filter state, the strain history, the running peaks and the
 * sample counter (enqueued on `stream`). */
spiir_status spiir_reset(spiir_plan *plan, void *stream);

/*
 * Filter the next n samples of every detector stream: the summed IIR bank of
 * subsection "SPIIR method", y_l[k] = a_l y_l[k-1] + b_l x[k - d_l] and
 * z[k] = sum_l y_l[k] for every (detector, template).
 *   x_dev  [n_detectors][n] float32, row stride n (detector-major)
 *   n      >= 0 samples (top rate for multirate banks)
 *   z_dev  [n_detectors][n_templates][n] complex64 output in the bank's
 *          template order, or NULL to skip storing z (the running peak is
 *          still updated).
 * Consecutive calls continue one stream: the result equals one call on the
 * concatenated samples (the plan keeps each filter's state and the last
 * history_len samples of strain).  Multirate banks: band j sees
 * x[R_j * k] (R_j = band_decim[j]) counted from the stream start, and its
 * summed output is linearly interpolated to the top rate; within one call
 * the samples after the last band sample use that sample (hold).  For
 * multirate banks every call's n must be a multiple of the largest R_j
 * except the last one.
 * Errors: EINVAL, ENOMEM (workspace growth), ECUDA.
 */
spiir_status spiir_filter(spiir_plan *plan, const float *x_dev, int64_t n, float *z_dev,
                          void *stream);

/*
 * Running peak of every (detector, template) since the last reset (the
 * largest |z|, which flags a candidate signal, subsection "SPIIR method"):
 *   peak_abs_dev [n_detectors][n_templates] float32  max_k |z[k]|
 *   peak_idx_dev [n_detectors][n_templates] int64    its absolute sample index
 *                                                    (top rate); ties keep the
 *                                                    earliest; -1 if no sample
 * |z|^2 is evaluated as re*re + im*im in float32 without fused multiply-add
 * and peak_abs is its correctly rounded square root.
 */
spiir_status spiir_peak(spiir_plan *plan, float *peak_abs_dev, int64_t *peak_idx_dev,
                        void *stream);

/*
 * Front end of one band (whitening and/or anti-aliasing before the band's
 * subsampling; section "SPIIR method" filters noisy detection data, which a
 * pipeline whitens first and brings to each band's rate): from the next
 * spiir_filter call on, band `band` (an index into the bank's bands) sees
 *   x_band[k] = sum_{i < n_taps} taps[i] x[R k - i]
 * (x at the top rate counted from the stream start, x[< 0] = 0, R the
 * band's decimation factor; R = 1 bands too) instead of x[R k].  The plan
 * keeps the last 511 top-rate samples for this across calls; spiir_reset
 * zeroes them.  FP32 products accumulated in tap order.
 *   taps    [n_taps] float32, host, copied
 *   n_taps  0 (plain subsampling again) .. 512
 * Waits for the plan's device work to finish.  spiir_state_set refuses
 * plans with front ends (EUNSUPPORTED): their history is not in the state.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
spiir_status spiir_set_band_fir(spiir_plan *plan, int32_t band, const float *taps,
                                int32_t n_taps);

/*
 * Chi^2 bins of every template of a bank (the review's chi^2 section: Allen's
 * discriminator compares the SNR collected by p frequency bins of equal
 * template power with each bin's share).  A SPIIR template is a sum over
 * frequency, one single-pole filter per stretch of the chirp, so a bin is a
 * contiguous run of a template's filters ordered by arg(a_l) (ties keep bank
 * order), and a filter's power is its impulse-response energy
 * |b_l|^2 / (1 - |a_l|^2).  Filter l joins bin floor(p m_l) (at most p - 1),
 * m_l being the midpoint of its share of the template's cumulative energy,
 * (cumulative energy up to and including l - half its own) / total, in
 * double precision; a template of zero energy goes to bin 0.  Bin i of
 * template t becomes template t * n_bins + i of the regrouped bank (empty
 * bins stay empty), its filters in frequency order.
 *   bank        host bank, as for spiir_plan_create (single-rate)
 *   n_bins      1 <= p <= 64
 *   group_off   [n_templates * n_bins + 1] int64, host, out: the regrouped
 *               bank's CSR offsets
 *   filter_of   [Ltot] int64, host, out: the bank filter at each position of
 *               the regrouped bank
 *   a_out, b_out [2 * Ltot] complex64, host, out (or NULL): its poles, gains
 *   delay_out   [Ltot] int32, host, out (or NULL): its delays
 * Host only (no device work, no allocation visible to the caller).
 * Errors: EINVAL (bad bank, n_bins, NULL outputs), EUNSUPPORTED (multirate).
 */
spiir_status spiir_chi2_split(const spiir_bank_desc *bank, int32_t n_bins, int64_t *group_off,
                              int64_t *filter_of, float *a_out, float *b_out,
                              int32_t *delay_out);

/*
 * Chi^2 signal-based veto at each template's peak (Allen's discriminator,
 * the review's chi^2 section).  Its p bins are groups of a template's
 * filters (contiguous in frequency, equal impulse-response energy;
 * spiir_chi2_split builds the regrouped bank), filtered as templates of
 * their own, so spiir_filter on the regrouped bank writes the group series
 * z_i in the layout read here.  Per (detector, template):
 * z = sum_i z_i (float32, group order), t = the first index maximising
 * |z|^2 (re*re + im*im, separately rounded products), peak = sqrt(|z(t)|^2)
 * (correctly rounded) and chi2 = p sum_i |z_i(t) - z(t) / p|^2 (raw z
 * units; for unit white noise its mean is (p - 1) times a bin's noise
 * power).
 *   zg_dev    [n_detectors][n_templates][n_bins][n] complex64, device
 *   peak_dev, chi2_dev  [n_detectors][n_templates] float32, device
 *   t_dev     [n_detectors][n_templates] int64, device
 * No plan; current device; asynchronous on `stream`.  1 <= n_bins <= 64,
 * n >= 1.  Errors: EINVAL, ECUDA.
 */
spiir_status spiir_chi2_peak(const float *zg_dev, int32_t n_detectors, int64_t n_templates,
                             int32_t n_bins, int64_t n, float *peak_dev, int64_t *t_dev,
                             float *chi2_dev, void *stream);

/*
 * Network peak across detectors (coincidence of the SNR series).  A signal
 * reaches the detectors at times that differ by at most their light travel
 * time; the review's multi-messenger section localises a source from these
 * arrival-time differences.  With detector 0 as the reference, per template
 *   s(t) = |z_0(t)|^2 + sum_{d>=1} max_{|u| <= window[d], 0 <= t+u < n} |z_d(t+u)|^2,
 * over t in [0, n), and returns the first t maximising s, rho = sqrt(s(t)),
 * and per detector d >= 1 the first offset u (from -window[d] upward) whose
 * |z_d(t+u)|^2 reaches that maximum.  |z|^2 = re*re + im*im with separately
 * rounded float32 products, the detector terms summed in detector order and
 * a correctly rounded sqrt, so t and the offsets are exact.
 *   z_dev      [n_detectors][n_templates][n] complex64, device (the layout
 *              spiir_filter writes)
 *   window     [n_detectors] int32, host; window[0] is ignored, others in
 *              [0, 1024] samples
 *   rho_dev    [n_templates] float32, device
 *   t_dev      [n_templates] int64, device (while the call runs it holds a
 *              per-template reduction key; its final contents are the t*)
 *   shift_dev  [n_templates][n_detectors] int32, device, or NULL (column 0 = 0)
 * No plan: works on any series of that layout, on the current device,
 * asynchronously on `stream` (one or two kernels and a memset).  1 <= n_detectors <= 8, n >= 1 (n_templates
 * = 0 is a no-op).
 * Errors: EINVAL, EUNSUPPORTED (windows too wide for shared memory), ECUDA.
 */
spiir_status spiir_network_peak(const float *z_dev, int32_t n_detectors, int64_t n_templates,
                                int64_t n, const int32_t *window, float *rho_dev,
                                int64_t *t_dev, int32_t *shift_dev, void *stream);

/*
 * Vector-Jacobian product of one spiir_filter call made from zero state on
 * x_dev (single-rate banks): the reverse-time (adjoint) recurrence of the
 * filter bank, lambda_l[k] = g_z[k] + conj(a_l) lambda_l[k+1], used when the
 * filter coefficients are fitted to a template (section "SPIIR method":
 * each template's filters are designed to reproduce its matched filter).  grad_z_dev [n_detectors][n_templates][n]
 * complex64 holds g_z = dL/dRe z + i dL/dIm z (the PyTorch convention);
 * outputs use the same convention and are OVERWRITTEN:
 *   grad_a_dev, grad_b_dev  [Ltot] complex64 (summed over detectors)
 *   grad_x_dev              [n_detectors][n] float32, or NULL
 * g_a and g_b (spiir_options.adjoint_form): the reverse form recomputes the
 * forward from state checkpoints kept in plan workspace and runs the adjoint
 * recurrence backwards in time; the tangent form runs, forward in time, each
 * filter's unit-gain response u_l[k] = a_l u_l[k-1] + x[k-d_l] and its
 * derivative recurrence v_l[k] = a_l v_l[k-1] + u_l[k-1], and sums
 * g_b_l = sum_k g_z[k] conj(u_l[k]), g_a_l = conj(b_l) sum_k g_z[k] conj(v_l[k])
 * (the same sums as sum_k lambda_l[k] x[k-d_l] and
 * sum_k lambda_l[k] conj(y_l[k-1]), in the other order).
 * grad_x is summed over filters in the shifted adjoint frame (each filter
 * reads g_z at its own delay, all meet at one output sample) and over
 * templates with float atomics, so its last bits depend on timing.
 * Does not touch the plan's streaming state.
 * Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED (multirate bank, or delays
 * whose adjoint windows exceed 227 KB of shared memory).
 */
spiir_status spiir_filter_backward(spiir_plan *plan, const float *x_dev, int64_t n,
                                   const float *grad_z_dev, float *grad_a_dev,
                                   float *grad_b_dev, float *grad_x_dev, void *stream);

/*
 * Replace every filter's pole and gain (device arrays, [Ltot] complex64 in
 * bank order, read on `stream`); delays and the layout are unchanged.  Used
 * when the coefficients are being fitted (see spiir_filter_backward).  The
 * caller keeps |a_l| < 1; the device values are not validated.
 */
spiir_status spiir_set_coefficients(spiir_plan *plan, const float *a_reim_dev,
                                    const float *b_reim_dev, void *stream);

/*
 * Streaming state, for checkpoint and resume.  Synchronous (waits for the
 * plan's device work).  Host buffers:
 *   state   [n_detectors][Ltot] complex64 filter outputs y_l at the last
 *           processed sample (multirate: at the last sample of its band)
 *   history [n_detectors][history_len] float32 last strain samples, oldest
 *           first (zeros before the stream start; single-rate banks)
 *   samples total samples processed since the last reset
 * Either array pointer may be NULL to skip it.
 */
spiir_status spiir_state_get(spiir_plan *plan, float *state, float *history,
                             int64_t *samples);
spiir_status spiir_state_set(spiir_plan *plan, const float *state, const float *history,
                             int64_t samples);

/*
 * Wait for the plan's work on `stream` and read its device error word.
 * Returns ETIMEOUT if a bounded device wait gave up since the last reset.
 */
spiir_status spiir_check(spiir_plan *plan, void *stream);

/*
 * Self-test of the bounded-wait path: launches one CTA that waits on an
 * mbarrier nothing completes, for at most limit_ns nanoseconds, then records
 * the timeout in the plan's error word (so spiir_check returns ETIMEOUT).
 * No kernel traps or hangs.
 */
spiir_status spiir_selftest_bounded_wait(spiir_plan *plan, uint64_t limit_ns, void *stream);

/*
 * One-shot filter call that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or cudaFree -- for instance a process whose device memory is
 * owned by another allocator or a fixed budget, or a low-latency pipeline
 * that must not allocate while it streams -- and therefore cannot create a
 * plan (spiir_plan_create allocates the packed parameters and workspace).
 *
 * It runs the plain FP32 kernel of spiir_filter, on the layout a default
 * plan would use, from zero state (no streaming, single-rate banks only),
 * and keeps all of its scratch (packed parameters, filter state, staged
 * strain, running peaks) in one static device array of 32 MiB that every
 * GPU loading this library holds until the process exits.
 *   bank          host bank description, as for spiir_plan_create
 *   x_dev         [n_detectors][n] float32 strain, 1 <= n <= 2^30
 *   z_dev         [n_detectors][n_templates][n] complex64 output, or NULL
 *   peak_abs_dev  [n_detectors][n_templates] float32 max |z|
 *   peak_idx_dev  [n_detectors][n_templates] int64 first index of the max
 * The call does not wait for its device work, so it cannot return
 * SPIIR_ETIMEOUT (spiir_check needs a plan): if a bounded device wait of the
 * call gave up, every peak_abs is NaN and every peak_idx -1, and z is
 * undefined.  A caller checks its peaks after synchronizing the stream.
 * Runs on the caller's current device and `stream`.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call reuses the same
 * array and clears what must start at zero; calls whose GPU work overlaps
 * (different streams, or different host threads, without ordering) race on
 * the array and must be serialized by the caller.
 * Errors: EINVAL (bad bank or sizes, or a problem needing more than the
 * 32 MiB of scratch -- the message gives the bytes needed), EUNSUPPORTED
 * (multirate bank, device not sm_103), ECUDA.
 */
spiir_status spiir_filter_noalloc(const spiir_bank_desc *bank, const float *x_dev, int64_t n,
                                  float *z_dev, float *peak_abs_dev, int64_t *peak_idx_dev,
                                  void *stream);

/* Device time of the kernels launched since the last read (plans created
 * with kernel_timing set; events recorded on the call's stream around each
 * launch).  Waits for the recorded events, sums their durations per kernel
 * class and clears the record.
 *   ms[SPIIR_KERNEL_CLASSES]  total milliseconds per class (host array)
 *   n[SPIIR_KERNEL_CLASSES]   launches per class (host array, may be NULL)
 * Classes: 0 the filter kernel (all K1 passes), 1 the tensor-core
 * projection, 2 the adjoint's kernels (its reverse pass or its tangent
 * pass, and its input-gradient pass with that pass's projection).
 * Errors: EINVAL (NULL plan or ms), ECUDA. */
#define SPIIR_KERNEL_CLASSES 3
spiir_status spiir_kernel_times(spiir_plan *plan, double *ms, int64_t *n);

/* Static description of a status code. */
const char *spiir_status_str(spiir_status status);

/* One-line reason for the last failure on this host thread ("" if none). */
const char *spiir_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* SPIIR_H */
