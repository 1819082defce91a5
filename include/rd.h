/*
 * rd.h -- C ABI of a GB300 (sm_103a) library for the spatiotemporal radiation deposit of
 * RaDiO (Pardal, Sainte-Marie, Reboul-Salze, Fonseca, Vieira: "RaDiO: an efficient
 * spatiotemporal radiation diagnostic for particle-in-cell codes").
 *
 * For every (particle, trajectory interval, detector cell) triple the library
 *   - evaluates the Lienard-Wiechert fields of Eq. 1 (velocity and acceleration terms) from the
 *     particle's position, beta = u/sqrt(1+u^2) and betadot = (beta_k - beta_{k-1})/dt
 *     (Algorithm 1);
 *   - computes the arrival time t_det = t_k + |x_k - x_cell| (Eq. 2, c = 1);
 *   - deposits E and B = n x E into the cell's time bins with the integrating interpolation of
 *     Section 3.2 / Algorithm 2: the field of sample k is held constant between the arrival
 *     times of samples k-1 and k, and bin b receives field * overlap / dt_det.
 *
 * Units: c = 1; momenta u = p/(m c) = gamma*beta; each particle carries a signed charge q (a
 * macro-particle radiates as one point charge N*q, Section 4.2); fields are q / length^2.
 *
 * Conventions for every call:
 *   - All entry points return an rd_status; nothing aborts.  rd_last_error() gives a message for
 *     the last failing call on the calling thread.
 *   - Work is enqueued on the caller's CUDA stream and is asynchronous unless stated otherwise.
 *   - Errors found by kernels (invalid trajectory samples, a bounded wait that ran out, an index
 *     outside the detector) are latched in the detector and returned by the next synchronising
 *     call (rd_read_fields to host memory, rd_get_stats, rd_synchronize).
 *   - A detector object may be used from one host thread at a time.
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RD_API __attribute__((visibility("default")))
#else
#define RD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t / CUstream).  NULL selects the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st* rd_stream;

/* Opaque detector: geometry, time axis, field accumulators and scratch; owned by the library. */
typedef struct rd_detector rd_detector;

typedef enum {
    RD_OK = 0,
    RD_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, bad enum value)           */
    RD_ERR_CUDA = 2,     /* a CUDA runtime call failed                                          */
    RD_ERR_OOM = 3,      /* device or pinned-host allocation failed                             */
    RD_ERR_STATE = 4,    /* call not valid for this detector (e.g. wrong precision)             */
    RD_ERR_TIMEOUT = 5,  /* a kernel's bounded wait ran out; its work was abandoned              */
    RD_ERR_BOUNDS = 6,   /* a kernel found an index outside the detector (internal error)       */
    RD_ERR_INPUT = 7     /* trajectory rejected: chord speed |x_k - x_{k-1}|/dt >= 1 or not finite */
} rd_status;

/* precision of a detector */
enum { RD_FP64 = 0, RD_MIXED = 1 };
/*
 * terms of Eq. 1 to evaluate (bit set); the default is both.  RD_FARFIELD (with RD_FAR, without
 * RD_NEAR) selects the far-field limit: arrival times by Eq. 3, t + R_c - x.n_c, and the radiation
 * term of Eq. 1 with the direction n_c and distance R_c of the cell seen from the origin
 * (R_c n_c = pix_pos) in place of the particle-to-cell n and R.
 *
 * RD_LINEAR (with any of the above) replaces the held field of the integrating deposit by a field
 * that varies linearly in arrival time over each interval, from the field of sample k-1 to that
 * of sample k (second order in dt where the held field is first order; the first interval of a
 * trajectory still holds the field of sample 1).  RD_HOLD_PREV (instead of RD_LINEAR) holds the
 * field of sample k-1 over interval k (the reading of Section 3.2's worked example, which writes
 * the field at the interval's start; first order like the default, which holds the field of
 * sample k as Algorithm 2 passes it); interval 1 holds the field of sample 1.  RD_QUADRATIC (instead
 * of the two) makes the field over interval k the quadratic in arrival time through the fields of
 * samples k-2, k-1 and k at their arrival times, integrated exactly over each bin overlap (third
 * order in dt); interval 2 is linear and interval 1 holds the field of sample 1 (the first samples
 * have fewer fields behind them).  None of the three is supported by rd_adjoint_trajectories.
 */
enum { RD_NEAR = 1, RD_FAR = 2, RD_FARFIELD = 4, RD_LINEAR = 8, RD_HOLD_PREV = 16, RD_QUADRATIC = 32 };
/* where a caller buffer lives; RD_MEM_HOST_ASYNC: pinned host memory written asynchronously
 * (rd_read_fields only) */
enum { RD_MEM_DEVICE = 0, RD_MEM_HOST = 1, RD_MEM_HOST_ASYNC = 2 };
/* element type of caller field / gradient-seed buffers */
enum { RD_F32 = 0, RD_F64 = 1 };
/* field whose power spectrum rd_power_spectrum computes */
enum { RD_SPEC_E = 0, RD_SPEC_B = 1 };

/*
 * Virtual detector (Section 3.1): n_pix cells at positions pix_pos, each with a uniform time
 * axis of n_bins bins; bin b of cell j covers
 *     [t_min + pix_t0[j] + b*dt_det,  t_min + pix_t0[j] + (b+1)*dt_det).
 * pix_t0 == NULL means 0 for every cell (one global time array as in the paper).
 * The arrays are read during rd_create_detector only (copied); `mem` says where they live.
 * precision: RD_MIXED -- fields and accumulation in FP32, arrival times FP64-accurate;
 *            RD_FP64  -- everything in FP64.
 */
typedef struct {
    int32_t n_pix;             /* >= 1                                                          */
    const double* pix_pos;     /* [n_pix][3]                                                    */
    const double* pix_t0;      /* [n_pix] or NULL                                               */
    int32_t mem;               /* RD_MEM_DEVICE or RD_MEM_HOST for pix_pos / pix_t0             */
    double t_min;
    double dt_det;             /* > 0                                                           */
    int32_t n_bins;            /* >= 1; <= 4194304 (2^22) for RD_MIXED                          */
    int32_t precision;         /* RD_MIXED or RD_FP64                                           */
    int32_t flags;             /* RD_NEAR | RD_FAR (0 = both), or RD_FAR | RD_FARFIELD;
                                  | RD_LINEAR, | RD_HOLD_PREV or | RD_QUADRATIC                   */
} rd_detector_desc;

/*
 * Trajectories (Algorithm 1 inputs): n_part particles, each with n_samples = S+1 samples at
 * t_k = t0 + k*dt, k = 0..S.  Interval k (1..S) lies between samples k-1 and k; sample 0 only
 * provides the previous position and velocity.  Layout [n_part][n_samples][3], row-major FP64.
 * q: [n_part] charges, or NULL for q = 1.  All three arrays live where `mem` says; host arrays
 * are copied to the device inside the call (pinned host memory copies asynchronously).
 * The caller keeps ownership and must keep the arrays alive until the stream has passed the call.
 */
typedef struct {
    int32_t n_part;            /* >= 0                                                          */
    int32_t n_samples;         /* >= 1 (S = n_samples - 1 intervals)                            */
    const double* x;           /* positions  [n_part][n_samples][3]                             */
    const double* u;           /* momenta gamma*beta [n_part][n_samples][3]                     */
    const double* q;           /* [n_part] or NULL                                              */
    int32_t mem;               /* RD_MEM_DEVICE or RD_MEM_HOST                                  */
    double t0;
    double dt;                 /* > 0                                                           */
} rd_traj;

/* Counters of a detector (rd_get_stats). */
typedef struct {
    int64_t n_clipped;         /* (particle, interval, cell) triples whose arrival interval had
                                  a part outside the cell's window (that part is dropped,
                                  Algorithm 1 window test read as clipping)                    */
    int64_t n_deposits;        /* triples processed since creation / last rd_zero_fields        */
    int64_t n_bin_crossings;   /* bin edges crossed by the arrival intervals (RD_MIXED): the
                                  deposit touched n_deposits + n_bin_crossings (cell, bin) pairs  */
    uint32_t device_errors;    /* bit set of latched kernel errors (1<<RD_ERR_*)               */
    int64_t kernel_launches;   /* deposit-kernel launches timed since the last rd_get_stats     */
    double kernel_ms;          /* their summed duration (CUDA events on the caller's stream)    */
} rd_stats;

/*
 * Create a detector and zero its fields.  Allocates device memory for the cell table and the
 * accumulators ([n_pix][n_bins] E and B: 32 bytes per bin in RD_MIXED, 48 in RD_FP64).
 * On success *out owns the detector (free with rd_destroy).  Errors: RD_ERR_ARG, RD_ERR_OOM,
 * RD_ERR_CUDA.  The device is the one current on the calling thread.
 */
RD_API rd_status rd_create_detector(const rd_detector_desc* desc, rd_stream stream, rd_detector** out);

/* Release every resource of the detector (synchronises its device work first).  NULL is a no-op. */
RD_API rd_status rd_destroy(rd_detector* det);

/* Set all fields and counters of the detector to zero (asynchronous). */
RD_API rd_status rd_zero_fields(rd_detector* det, rd_stream stream);

/*
 * Deposit the radiation of the given trajectories: ACCUMULATES (+=) into the detector, so a run
 * can be split over particle chunks or over step chunks that share one sample (the last sample
 * of chunk i is sample 0 of chunk i+1; the run-time mode of Section 3.1).
 * Uses Eq. 1, Eq. 2 and the integrating deposit of Section 3.2 for every (particle, interval,
 * cell) triple.  Scratch for per-sample records is kept in the detector and grown as needed.
 * Errors: RD_ERR_ARG (bad sizes or pointers), RD_ERR_OOM, RD_ERR_CUDA; invalid samples are
 * reported as RD_ERR_INPUT by the next synchronising call (their deposits are undefined).
 */
RD_API rd_status rd_deposit_trajectories(rd_detector* det, const rd_traj* traj, rd_stream stream);

/*
 * Copy the accumulated fields out as E[n_pix][n_bins][3] and B[n_pix][n_bins][3] (either may be
 * NULL) of type dtype (RD_F32 / RD_F64) into memory of kind mem.  To host memory (RD_MEM_HOST)
 * the call synchronises the stream and then reports latched kernel errors; to device memory it is
 * asynchronous.  RD_MEM_HOST_ASYNC: E and B are page-locked host memory (cudaHostAlloc or
 * registered); the layout conversion and the device-to-host copies are enqueued on the stream and
 * the call returns at once, so that a caller can enqueue the next deposit (on another detector and
 * stream) behind them and overlap the copies with its kernel.  The host buffers are complete once
 * the stream has been synchronised (rd_synchronize then reports latched errors); the detector's
 * readback scratch is reused by its next read, which must come after that.  Errors: RD_ERR_ARG,
 * RD_ERR_CUDA, RD_ERR_OOM, latched errors.
 */
RD_API rd_status rd_read_fields(rd_detector* det, void* E, void* B, int32_t dtype, int32_t mem,
                         rd_stream stream);

/*
 * Set the detector's accumulated fields to E[n_pix][n_bins][3] and B[n_pix][n_bins][3] (the layout
 * rd_read_fields writes; dtype RD_F32 or RD_F64, converted to the detector's precision; either may
 * be NULL, which sets that part to zero).  Deposits add (the detector holds the superposition of
 * everything deposited, Section 3.2), so a run checkpointed with rd_read_fields resumes in a new
 * detector (or process) by rd_write_fields followed by the remaining deposits: particle subsets
 * and step chunks that share their boundary sample, as the run-time mode of Section 3.1 hands
 * them over (exact for the held field; an interpolated field restarts its first interval).
 * Counters and the state of streamed deposits are not part of the fields and are left alone.
 *   mem: RD_MEM_DEVICE (device pointers, asynchronous), RD_MEM_HOST (any host memory; the call
 *        returns after the copy), RD_MEM_HOST_ASYNC (pinned host memory the caller keeps until the
 *        stream has passed the call).  Host input is staged in the detector's readback buffer, so
 *        it must not overlap a host readback of the same detector enqueued on another stream.
 * Errors: RD_ERR_ARG (NULL detector, bad dtype or mem), RD_ERR_OOM (staging for host input),
 * RD_ERR_CUDA.
 */
RD_API rd_status rd_write_fields(rd_detector* det, const void* E, const void* B, int32_t dtype, int32_t mem,
                                 rd_stream stream);

/*
 * Streamed deposit (Section 3: run-time use inside a particle code, which hands over each new
 * stretch of the trajectories as it computes them).  traj holds the NEW samples only, at
 * t0 + k*dt, k < n_samples; the detector keeps every particle's last sample from the previous
 * streamed call and deposits the interval from it to the first new sample, so that consecutive
 * calls on consecutive, non-overlapping stretches deposit exactly what one call on the whole
 * trajectory would (up to FP32 summation order and, in RD_MIXED, the placement of the FP64
 * arrival-time anchors).  The first call after creation or rd_stream_reset has nothing in front
 * of its first sample (as in rd_deposit_trajectories).  A continuing call must have the same
 * n_part and dt, and t0 equal to the stored last time + dt; otherwise RD_ERR_STATE.  With RD_LINEAR
 * the detector keeps the last two samples (the field of the last one needs its betadot), so every
 * stretch's first interval is interpolated like the others.  Memory: the
 * new samples are copied (host or device) behind the stored ones into detector-held scratch,
 * 48 bytes per particle and sample.  Each call pays a record precompute, a launch and FP64 arrival
 * anchors at both ends of its stretch: hand over several steps per call where the caller can.
 * Asynchronous on `stream`; calls of one stream must come in order on one CUDA stream.
 */
RD_API rd_status rd_deposit_stream(rd_detector* det, const rd_traj* traj, rd_stream stream);

/* Forget the stored last samples: the next rd_deposit_stream call starts a new stream. */
RD_API rd_status rd_stream_reset(rd_detector* det);

/*
 * Power spectrum of every cell's time series (Section 4: the detector data Fourier transformed in
 * time, the spectra compared with Eq. 8 and Eq. 9).  With N = n_bins, F = E (which = RD_SPEC_E) or
 * B (RD_SPEC_B) and F_c[j][b] the bin values:
 *     out[j][k] = dt_det^2 * sum_{c=x,y,z} | sum_{b<N} F_c[j][b] exp(-2 pi i k b / N) |^2,
 * k = 0..N/2, angular frequency w_k = 2 pi k / (N dt_det).  The bins are averages over dt_det,
 * so the spectrum of the underlying field is out / sinc^2(w dt_det / 2) below the Nyquist
 * frequency.  out: caller-owned device memory, float[n_pix][N/2 + 1].  FP32 FFT (relative error
 * ~1e-6 of the spectrum's norm).  Requires N a power of two (else RD_ERR_ARG); scratch of
 * 32 * n_pix * N bytes held by the detector.  Asynchronous on `stream`.
 */
RD_API rd_status rd_power_spectrum(rd_detector* det, int32_t which, float* out, rd_stream stream);

/* Synchronise the stream and return (then clear) latched kernel errors. */
RD_API rd_status rd_synchronize(rd_detector* det, rd_stream stream);

/* Synchronise the stream and fill *out with the detector's counters (does not clear errors).
 * kernel_launches / kernel_ms cover the deposit kernels timed since the previous call (then reset). */
RD_API rd_status rd_get_stats(rd_detector* det, rd_stream stream, rd_stats* out);

/* Enable (1) or disable (0) timing of every deposit-kernel launch with a pair of CUDA events
 * recorded on the launch stream around it (read back through rd_get_stats). */
RD_API rd_status rd_set_timing(rd_detector* det, int32_t enable);

/*
 * Adjoint (gather) form of rd_deposit_trajectories, for gradients of a scalar loss L(E_det, B_det).
 * gE, gB: d L / d E_det and d L / d B_det, [n_pix][n_bins][3] of type gdtype (RD_F32/RD_F64) in
 * device memory; either may be NULL (zero).  Accumulates (+=) d L / d x into gx and d L / d u
 * into gu, both [n_part][n_samples][3] FP64 in device memory, for the deposit this detector would
 * make from `traj` (same windows, flags and arithmetic as its forward path of the same precision).
 * The transpose of the integrating deposit (Section 3.2) per (particle, interval, cell): the seed
 * gathered over the bins the arrival interval covers drives the derivative of Eq. 1 (field of the
 * interval's sample); the bins at the two ends of the interval move with the arrival times of
 * Eq. 2, contributing (F_k - F_{k+1}) . g at each sample's arrival bin; beta = u/sqrt(1+u^2) and the
 * backward difference betadot couple neighbouring samples.  Nothing per triple is stored: the
 * forward quantities are recomputed from x and u.  RD_MIXED: FP32 field arithmetic with the
 * forward path's FP32 arrival-time walk, restarting from exact FP64 arrival times every 250
 * samples, FP64 gradient sums across cells (relative error ~1e-5, set by FP32 rounding in the
 * differences of neighbouring samples).  The derivative through an arrival time takes the seed of
 * the bin that arrival lies in; where the FP32 walk ends within 1e-4 bin of an edge (its drift is
 * ~1e-5 bin) that bin is taken from Eq. 2 in FP64.  RD_FP64: everything in FP64, Eq. 2 for every
 * sample (the plain form; relative error ~1e-12 against the exact derivative, at the FP64 rate of
 * the GPU).
 * Requirements: flags without RD_FARFIELD, RD_LINEAR and RD_HOLD_PREV (else RD_ERR_STATE), traj->mem
 * RD_MEM_DEVICE (else RD_ERR_ARG).
 */
RD_API rd_status rd_adjoint_trajectories(rd_detector* det, const rd_traj* traj, const void* gE,
                                         const void* gB, int32_t gdtype, double* gx, double* gu,
                                         rd_stream stream);

/*
 * Arithmetic of rd_adjoint_trajectories on an RD_MIXED detector.
 *   RD_ADJ_FP32 (default): FP32 field arithmetic (relative error ~1e-5, see above).
 *   RD_ADJ_COMPENSATED: the same gradient carried in double-float -- pairs of FP32 numbers, about
 *     48 significant bits, from FP32 operations only -- wherever a difference of neighbouring
 *     samples would magnify rounding: the field of Eq. 1, the seed gathered over each interval's
 *     bins (Section 3.2), the vector-Jacobian product up to d L / d beta and d L / d betadot, the
 *     projection to d L / d u, the arrival-time walk (the all-positive increment from an FP64
 *     arrival time of Eq. 2 at the start of every 250-sample chunk) and the sums over cells.  The
 *     two terms of each difference are formed in one thread (each chunk walks the interval before
 *     it once more).  Only the position derivative through the field's n and R (1/R of the
 *     others) stays FP32.  Relative error ~1e-8 against the exact derivative; several times the
 *     FP32 adjoint's time, several times faster than the RD_FP64 adjoint on this GPU's FP64 rate.
 *     Records of 128 bytes per particle and sample.
 * RD_ERR_ARG for an unknown mode, RD_ERR_STATE for RD_ADJ_COMPENSATED on an RD_FP64 detector.
 */
enum { RD_ADJ_FP32 = 0, RD_ADJ_COMPENSATED = 1 };
RD_API rd_status rd_set_adjoint_mode(rd_detector* det, int32_t mode);

/*
 * Batched form: deposit trajs[i] into dets[i] for i < n (ACCUMULATES, like n calls of
 * rd_deposit_trajectories) with one persistent kernel launch.  The resident CTAs draw work items
 * -- (problem, step chunk, block of 256 cells, particle) -- from one atomic counter, so problems of
 * very different size share the GPU without a tail of idle SMs; no CTA ever waits on another.
 * On a non-default stream the counter reset, the per-problem record precompute and the launch
 * are recorded once into a CUDA graph that is replayed while the same detectors (by identity),
 * trajectory pointers, shapes, time axes, chunks and flags come back; the graph reads the
 * trajectory arrays at replay time.  Every detector must be RD_MIXED and every trajectory in
 * device memory; the batch scratch and the graph live in dets[0].  Memory: the per-sample records
 * (64 bytes per particle and sample) are computed for a group of problems -- a problem's particles
 * may be split across groups -- whose records fit dets[0]'s batch budget (rd_set_batch_budget,
 * default 4 GiB); the groups run one after another, each as record precomputes plus one
 * persistent launch, reusing one record buffer.  Results equal the separate deposits up to FP32
 * summation order.
 */
RD_API rd_status rd_deposit_batch(int32_t n, rd_detector* const* dets, const rd_traj* trajs,
                                  rd_stream stream);

/*
 * Bytes of per-sample records per launch group of rd_deposit_batch calls whose first detector is
 * `det` (0 = the default, 4 GiB; a group always holds at least one particle).  No counterpart in
 * the paper: it bounds the batch scratch.  RD_ERR_ARG for a negative value.
 */
RD_API rd_status rd_set_batch_budget(rd_detector* det, long long bytes);

/*
 * Steps per work item (the step chunk between exact FP64 arrival anchors) for this detector's
 * deposits; 0 = automatic (2048, halved while the grid would be too small to fill the GPU).
 */
RD_API rd_status rd_set_chunk(rd_detector* det, int32_t chunk);

/*
 * Autotuner: time rd_deposit_trajectories of `traj` with step chunks 64, 128, ..., 4096 (up to
 * the trajectory length), keep the fastest for this detector (as rd_set_chunk) and return it in
 * *chosen.  The trial deposits go into this detector; its fields are zeroed afterwards.
 * Synchronises the stream.
 */
RD_API rd_status rd_autotune(rd_detector* det, const rd_traj* traj, rd_stream stream, int32_t* chosen);

/*
 * Launch shape of an RD_MIXED detector's deposit (no counterpart in the paper: how the (particle,
 * interval, cell) triples are split over the GPU).  A work item is one particle, one chunk of
 * intervals between FP64 arrival anchors and one block of cells_per_cta cells (the pixel strip),
 * walked by cells_per_cta / cells_per_thread threads; work items are ordered so that `group` cell
 * blocks take each particle back to back (its records then come from DRAM once per group).
 *   cells_per_cta    64, 128 or 256 (default 256)
 *   cells_per_thread 1 or 2 (default 2)
 *   chunk            intervals per work item, >= 0 (0: automatic, 2048 halved while the grid would
 *                    leave the GPU idle)
 *   group            cell blocks per group, >= 0 (0: automatic, as many as keep the group's active slice
 *                    of the detector -- cells_per_cta x 32 bytes x the bins one chunk's arrivals span,
 *                    taken as 1.25 x its share of the trajectory's bins, each -- within 70 MB of L2,
 *                    at most 8)
 * The far-field limit and the interpolation variants run the default cells per CTA and per thread
 * (their chunk and group follow the shape).  rd_deposit_batch uses every detector's chunk and group
 * and the default cells per CTA and per thread.  Results do not depend on the shape beyond the
 * order of FP32 reductions and the placement of the FP64 anchors.
 */
typedef struct {
    int32_t cells_per_cta;
    int32_t cells_per_thread;
    int32_t chunk;
    int32_t group;
} rd_shape;

/* Set / read the shape (RD_ERR_ARG for an unsupported one; RD_ERR_STATE on an RD_FP64 detector for
 * rd_set_shape).  rd_set_chunk(det, c) is rd_set_shape with only the chunk changed. */
RD_API rd_status rd_set_shape(rd_detector* det, const rd_shape* shape);
RD_API rd_status rd_get_shape(const rd_detector* det, rd_shape* shape);

/*
 * Shape autotuner: pick the fastest shape for depositing `traj` into this RD_MIXED detector and keep it
 * (as rd_set_shape).  With cache_path (a JSON file; NULL: no cache) an entry for the same device and
 * problem -- cells, bins, particles, intervals and flags -- is taken without timing (*from_cache = 1);
 * otherwise the tuner times rd_deposit_trajectories of `traj` (each candidate once after a warm-up,
 * CUDA events on `stream`) over every compiled cells-per-CTA x cells-per-thread shape at automatic
 * chunk and group, then the chunks 512 ... 4096 at the best shape, then the groups 1, 2, 4, 8, and adds
 * the winner to the cache file (read whole, rewritten whole through a temporary file).  The trial
 * deposits go into this detector, whose fields are zeroed afterwards.  Synchronises the stream.
 * chosen, from_cache and ms (the winner's time per deposit, or the cached one) may be NULL.
 * Errors: as rd_deposit_trajectories; RD_ERR_STATE on an RD_FP64 detector; RD_ERR_ARG for a cache
 * file that exists but cannot be read, parsed or written.
 */
RD_API rd_status rd_autotune_shape(rd_detector* det, const rd_traj* traj, const char* cache_path,
                                   rd_stream stream, rd_shape* chosen, int32_t* from_cache, double* ms);

/*
 * Allocation-free deposit.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc -- a particle-in-cell code that reserves all device memory in its
 * own pool at start-up and allows no allocation inside its time-step loop, a host framework whose
 * allocator owns the device memory, or a latency-bound loop that must not pay the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  It performs the same computation as
 * rd_deposit_trajectories on an RD_MIXED detector (Eq. 1, Eq. 2, integrating deposit; FP32 fields
 * and accumulation, FP64-anchored arrival times) without a detector object and without any
 * allocation: it calls no cudaMalloc, cudaFree or allocating library routine.
 *   pix_pos [n_pix][3], pix_t0 [n_pix] or NULL: cell positions and time origins (device memory);
 *     bin b of cell j covers [t_min + pix_t0[j] + b*dt_det, ... + dt_det); flags as RD_NEAR/RD_FAR.
 *   traj: trajectories in device memory (RD_MEM_DEVICE), as for rd_deposit_trajectories.
 *   fields: caller-allocated device accumulators float[n_pix][n_bins][8], per bin
 *     (Ex, Ey, Ez, Bx, By, Bz, unused, unused); the call ACCUMULATES (+=) into them.
 *   errors: NULL, or a host pointer that receives this call's latched kernel error bits
 *     (1 << RD_ERR_INPUT for a rejected sample or a cell with a non-finite position or time origin);
 *     given, the call synchronises the stream.  With errors == NULL the bits are not reported to
 *     anyone: the next call clears them before it starts.
 *   flags are checked as rd_create_detector checks them (RD_ERR_ARG for a set that selects no term
 *     of Eq. 1, e.g. RD_LINEAR or RD_FARFIELD alone).
 * Scratch: one 64 MiB array inside the library, held by every GPU that loads it until the process
 * exits.  Limits: n_pix <= 262144, n_bins <= 4194304, and one particle's samples must fit the 56 MiB record area
 * (n_samples <= 917500); larger requests return RD_ERR_ARG.  Particles are processed in chunks
 * that fit.  The first call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture.  Every call shares the array, which keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Asynchronous on `stream` unless `errors` is given.
 */
RD_API rd_status rd_deposit_noalloc(const double* pix_pos, const double* pix_t0, int32_t n_pix,
                                    double t_min, double dt_det, int32_t n_bins, int32_t flags,
                                    const rd_traj* traj, float* fields, uint32_t* errors,
                                    rd_stream stream);

/*
 * Run-time coupling (Section 3.1: the deposit runs as a sub-step right after the particle push,
 * from the new positions and momenta and the stored previous ones).  Advances n_part charges by
 * n_steps Boris steps of dt in a uniform magnetic field B[3] (host array; c = 1, qm = charge to mass
 * ratio, the same for every particle): t = (qm dt / 2) B / gamma, s = 2 t / (1 + |t|^2),
 * u' = u + u x t, u <- u + u' x s, x <- x + dt u / gamma (|u|, hence gamma, is kept; u turns about
 * B by 2 atan(|t|) per step).  x, u: the state [n_part][3] FP64 in device memory, updated in place.
 * x_out, u_out: [n_part][n_steps][3] FP64 in device memory, the new samples (after a state at time
 * t, sample k is at t + (k + 1) dt), laid out as rd_deposit_stream takes a stretch of new samples.
 * Asynchronous on `stream`.  RD_ERR_ARG for a negative count, a NULL pointer or a non-finite dt,
 * qm or field.
 */
RD_API rd_status rd_push_boris(int32_t n_part, int32_t n_steps, double dt, const double* B, double qm,
                               double* x, double* u, double* x_out, double* u_out, rd_stream stream);

/*
 * Diagnostic, not part of the deposit: the FP32 and FP64 fused multiply-add throughput of the
 * current device, measured by a microbenchmark (independent FMA chains on every SM, one launch
 * of about 20 ms per precision, timed with CUDA events on `stream`).  These are the denominators
 * of the roofline of the deposit kernels, which are bound by FP32 (RD_MIXED) and FP64 (RD_FP64)
 * arithmetic.  Results in TFLOP/s (one FMA = 2 flops); either pointer may be NULL to skip that
 * precision.  Synchronous; allocates and frees a few KB of device memory.
 */
RD_API rd_status rd_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, rd_stream stream);

/*
 * Diagnostic, not part of the deposit: checks the failure path of the kernels' bounded waits.
 * One CTA waits, with the same bounded mbarrier wait the deposit and adjoint kernels use for their
 * staged records, on a phase that nothing completes; after limit_ms (1..2000) the wait gives up,
 * the CTA records the expiry as those kernels do and returns, and this call reports it.
 * Returns RD_ERR_TIMEOUT when the expiry was detected and reported (the expected outcome; the
 * device stays usable), RD_ERR_STATE if it was not, RD_ERR_ARG for a limit outside the range,
 * RD_ERR_CUDA if a CUDA call failed.  Synchronous on `stream`.
 */
RD_API rd_status rd_check_bounded_wait(int32_t limit_ms, rd_stream stream);

/* Message for the last failing call on this thread ("" if none).  Valid until the next call. */
RD_API const char* rd_last_error(void);

/* Library version string. */
RD_API const char* rd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RD_H */
