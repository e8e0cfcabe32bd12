/*
 * wct_sim.h — C ABI of the GB300 (sm_103a) LArTPC signal-simulation hot path.
 *
 * The library implements the three steps of the Wire-Cell signal simulation described in
 * arXiv 2304.01841, §2 ("LArTPC Signal Simulation in the Wire-Cell Toolkit"):
 *   1. Rasterization: each drifted ionisation-electron group (a "depo") is binned into a
 *      patch of O(20x20) time-tick x pitch-impact bins (§2, item 1);
 *   2. Scatter-add: the patches are summed onto the plane's wire x tick grid (§2, item 2);
 *   3. Convolution: the grid is convolved with the 2D detector response by FFT (§2, item 3).
 * All three run in hand-written CUDA kernels; the caller owns the depo arrays, grids and
 * waveforms (device memory), the library owns the response spectra and its scratch.
 *
 * Conventions shared by every entry point:
 *  - Units: mm, microseconds, electrons.  Output waveforms are in (response units) x e-.
 *  - Device pointers are CUDA global-memory addresses on the current device; host pointers
 *    appear only where stated.  `stream` is a cudaStream_t (NULL = legacy default stream);
 *    every call is asynchronous on it unless stated otherwise.
 *  - Grids and waveforms are row-major float32 [n_wires][n_ticks] (ticks contiguous).
 *  - Argument errors are detected on the host and returned before anything is launched.
 *    Errors found by kernels (invalid depos, exceeded limits, timed-out waits) are recorded
 *    in a device status word and returned by wct_sim_sync() (or the next synchronising
 *    call).  The library never aborts, traps or exits; wct_sim_last_error() describes the
 *    most recent failure.
 *  - A handle is not thread-safe: use one handle per host thread or lock around it.  Its
 *    calls share the handle's device scratch, so enqueue them on one stream (or order the
 *    streams); wct_sim_run_host orders itself after all earlier device work.
 */
#ifndef WCT_SIM_H
#define WCT_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wct_sim wct_sim_t;   /* opaque, library-owned */

typedef enum {
    WCT_OK = 0,
    WCT_EINVAL = 1,     /* bad argument, or (device) invalid depo / depo window over the limits */
    WCT_ENOMEM = 2,     /* device allocation failed or would exceed the HBM budget */
    WCT_ECUDA = 3,      /* a CUDA runtime call failed */
    WCT_ETIMEOUT = 4,   /* a bounded device-side wait ran out */
    WCT_EBUSY = 5,      /* the handle is in use (e.g. during graph capture) */
    WCT_EDEVICE = 6     /* other device-side error */
} wct_status_t;

/* Largest depo window accepted (ticks x impact bins); a depo whose +-nsigma window is
 * larger is invalid (skipped and reported as WCT_EINVAL by wct_sim_sync). */
#define WCT_MAX_WINDOW_TICKS 128
#define WCT_MAX_WINDOW_IMPACTS 512
/* Largest response extent in wires (odd) handled by the wire stage. */
#define WCT_MAX_RESPONSE_WIRES 21

/*
 * One wire plane (§2: the "larger grid that spans the longitudinal time and transverse
 * space").  Wire w covers pitch coordinate [pitch_origin + w*pitch, +pitch); impact bin j
 * covers [pitch_origin + j*pitch/n_impact_per_pitch, ...) and folds onto wire
 * floor(j / n_impact_per_pitch).  Tick k covers [t_window0 + k*tick, +tick).  The pitch
 * coordinate of a point is p = z*cos(wire_angle) + y*sin(wire_angle).
 */
typedef struct {
    int32_t n_wires;
    int32_t n_impact_per_pitch;
    int32_t n_ticks;
    double pitch_mm;
    double pitch_origin_mm;
    double wire_angle_rad;
    double tick_us;
    double t_window0_us;
} wct_plane_t;

/*
 * Detector response of one plane (§2: "detector response with dimensions O(100x100)").
 * host_data: HOST pointer, row-major float32 [n_wires_resp][n_ticks_resp]; row
 * n_wires_resp/2 is the wire the charge arrives on, tick 0 is the arrival tick.
 * n_wires_resp must be odd and <= WCT_MAX_RESPONSE_WIRES.  Copied at create.
 */
typedef struct {
    int32_t n_wires_resp;
    int32_t n_ticks_resp;
    const float *host_data;
} wct_response_t;

/*
 * Drift / diffusion / fluctuation (the standard LArTPC picture behind §2's "individual
 * ionization electron groups"): drift time t_d = x / v_drift; longitudinal and transverse
 * widths sqrt(2 D t_d); patches span +-nsigma.  fluctuate != 0 draws a binomial-like
 * normal fluctuation per patch bin from a Philox4x32-10 stream keyed by `seed` (§4.1 names
 * Random123's Philox family as the CPU RNG) and renormalises each patch to its charge.
 */
typedef struct {
    double DL_cm2_s;
    double DT_cm2_s;
    double v_drift_mm_us;
    double nsigma;
    int32_t fluctuate;
    uint64_t seed;
} wct_diffusion_t;

/*
 * Library options.  hbm_budget_bytes: upper bound on the library's own device memory
 * (0 = unlimited); a call whose scratch would exceed it returns WCT_ENOMEM.
 * schedule_id: kernel-schedule choice, kept per handle.  -1 = the library's default
 * (paired row transforms with composite radices, warp-level rasterizer).  Otherwise a bit set:
 * row transforms 0 register-staged, 1 one persistent CTA per SM, 4 two paired CTAs per SM,
 * 8 paired with composite radices; +2 selects the CTA-level rasterizer.
 * deterministic: 0 = the scatter-add sums in float32 with atomics, so the last bits of a grid
 * bin can depend on the order in which contributions land (warp scheduling); 1 = bitwise
 * reproducible: every contribution is rounded to fixed point (2^-20 electrons) and summed as a
 * 64-bit integer, which is order independent, then converted once to float32 (the sum is exact
 * to 2^-21 electrons per contribution, finer than float32 at any bin above 8 electrons).  The
 * waveforms are then identical run to run, alone or in a batch, and for any order of the depos
 * when fluctuation is off (the fluctuation is keyed by depo index).  Costs 8 bytes of device
 * memory per grid bin per grid set (twice the float grids; the impact mode's phase grids
 * likewise) and a conversion pass over the touched tiles; forces the warp-level rasterizer.
 */
typedef struct {
    size_t hbm_budget_bytes;
    int32_t schedule_id;
    int32_t deterministic;
} wct_opts_t;

/*
 * One event's depos, structure of arrays in DEVICE memory (float32, n entries each):
 * t0 (us), x (drift distance, mm, >= 0), y, z (mm), q (electrons, >= 0).  The depo's
 * index in these arrays and event_id (low 24 bits) key its fluctuation counters.
 */
typedef struct {
    const float *t0_us;
    const float *x_mm;
    const float *y_mm;
    const float *z_mm;
    const float *q_e;
    int64_t n;
    uint64_t event_id;
} wct_depos_t;

/* Create a simulator for n_planes planes (1..8), each with its own response.  Builds the
 * FFT plans, uploads the responses and computes their spectra on the device (synchronous).
 * opts may be NULL (defaults).  On success *out receives the handle. */
wct_status_t wct_sim_create(const wct_plane_t *planes, int n_planes, const wct_response_t *responses,
                            const wct_diffusion_t *diffusion, const wct_opts_t *opts, wct_sim_t **out);

/* Free the handle and all library-owned device memory (synchronises the device). */
wct_status_t wct_sim_destroy(wct_sim_t *sim);

/*
 * Rasterization alone (§2 step 1), writing every depo's full patch.
 * patch_desc: DEVICE int64 [n][5] = {offset, lo_tick, lo_impact, n_ticks, n_impacts}; the
 *   offsets are the exclusive prefix sum of the patch sizes (the paper's scan, §4.3).
 *   Invalid depos get an empty window.
 * total_bins: HOST int64, receives the patch-buffer size (this call synchronises `stream`
 *   to read it back).
 * patches: DEVICE float32 [capacity], row-major [tick][impact] per patch, or NULL to only
 *   compute patch_desc / total_bins.  If total_bins > patches_capacity nothing is written
 *   to patches and WCT_EINVAL is returned.
 */
wct_status_t wct_sim_rasterize(wct_sim_t *sim, int plane, const wct_depos_t *depos, float *patches,
                               int64_t patches_capacity, int64_t *patch_desc, int64_t *total_bins,
                               void *stream);

/* Scan-free variant of wct_sim_rasterize (the paper's OpenMP port, §3.3, drops the prefix sum
 * for a fixed patch slot per depo at a small memory cost): depo i's patch, row-major
 * [tick][impact], is written at patches + i * slot_bins and patch_desc row i gets offset
 * i * slot_bins, so there is no size query and no host synchronisation.  patches: DEVICE
 * float32 of n * slot_bins; patch_desc: DEVICE int64 [n][5] as for wct_sim_rasterize.
 * 1 <= slot_bins <= 128 * 512.  A depo whose window holds more than slot_bins bins is skipped
 * (its descriptor row reads nt = np = 0) and reported as WCT_EINVAL at the next sync. */
wct_status_t wct_sim_rasterize_fixed(wct_sim_t *sim, int plane, const wct_depos_t *depos, float *patches,
                                     int64_t slot_bins, int64_t *patch_desc, void *stream);

/* The fixed patch slot of wct_sim_rasterize_fixed for depos that drift at most x_max_mm: the
 * bins of the largest +-nsigma window such a depo can have on `plane` (§2 item 1's patch,
 * §3.3's fixed slot).  The widths grow with the drift distance, sigma = sqrt(2 D x / v), so the
 * widest windows are those at x_max; per axis the window rule (bins overlapping
 * [mu - n sigma, mu + n sigma]) gives at most floor(2 n sigma) + 2 bins (1 for a point charge),
 * capped at the largest valid window (WCT_MAX_WINDOW_TICKS x WCT_MAX_WINDOW_IMPACTS).
 * *slot_bins (HOST int64) receives the product of the two extents.  Host computation in FP64
 * with the rasterizer's own expressions; no device work.  WCT_EINVAL for a NULL output or a
 * negative / non-finite x_max_mm. */
wct_status_t wct_sim_patch_slot_bins(wct_sim_t *sim, int plane, double x_max_mm, int64_t *slot_bins);

/*
 * Scatter-add onto the plane grid (§2 step 2).  grid: DEVICE float32 [n_wires][n_ticks],
 * fully overwritten (no need to clear it).  With patches == NULL the patches are computed
 * on the fly from `depos` (fused rasterize + scatter; patch_desc unused); otherwise
 * `patches` / `patch_desc` from wct_sim_rasterize are summed.  Patch bins outside the grid
 * are dropped.
 */
wct_status_t wct_sim_scatter(wct_sim_t *sim, int plane, const wct_depos_t *depos, const float *patches,
                             const int64_t *patch_desc, float *grid, void *stream);

/*
 * Convolution with the plane's response (§2 step 3):
 *   waveform[w][t] = sum_r sum_tau grid[w - (r - n_wires_resp/2)][t - tau] * resp[r][tau]
 * (linear, grid zero outside its extent, output cropped to the grid).  grid and waveform
 * are DEVICE float32 [n_wires][n_ticks] and may be the same buffer.
 */
wct_status_t wct_sim_convolve(wct_sim_t *sim, int plane, const float *grid, float *waveform, void *stream);

/* The whole DepoTransform (§2, all three steps) for every plane of one event.
 * waveforms: HOST array of n_planes DEVICE pointers, each float32 [n_wires][n_ticks].
 * The planes are rasterized one after the other on `stream`.  When `stream` has a priority
 * above the device's lowest (the default priority, 0, is the lowest), the event has two or
 * more planes, none in the impact mode, and stage timing is off, plane p's convolution runs
 * on a library stream of `stream`'s priority (two per priority, p mod 2) once that plane's
 * raster is done, while `stream` goes on with the next plane; `stream` waits for both before
 * later work.  Otherwise every step runs on `stream`: work on the lowest-priority stream is
 * treated as background work that should not occupy more of the GPU at once.  The second
 * stream's spectrum scratch is allocated at the first such call and counted against the HBM
 * budget; if it cannot be had, or with timing on, the planes run entirely on `stream`. */
wct_status_t wct_sim_run_event(wct_sim_t *sim, const wct_depos_t *depos, float *const *waveforms,
                               void *stream);

/* Several events in one pass: events[e] for e < n_events; waveforms: HOST array of
 * n_events * n_planes DEVICE pointers, event-major.  ONE persistent launch rasterizes and
 * scatters every plane of every event (§2 steps 1-2), each event into a library grid set of
 * its own: its warps take 8-depo chunks from a device counter, the largest events' chunks
 * first, until none is left.  The grids are then convolved (§2 step 3) on two library streams
 * taking the (event, plane) pairs alternately, each into the caller's waveform.  The grid sets
 * (every plane's grid per event, kept all zero between uses) are library memory grown on the
 * first call of a given size and counted against the HBM budget; if they do not all fit, the
 * batch runs in chunks of events, one raster launch per chunk, the raster of chunk c + 1
 * overlapping the convolutions of chunk c (schedule_id bits 4-7 ask for such chunks: value v
 * > 0 means 2^(v-1) events per launch; bit 8 selects a single convolution stream, bit 9 three).  All library
 * streams are ordered after earlier work on `stream`, and `stream` waits for them before
 * later work.  They are created at the first call: the rasterize stream with the priority of
 * that call's `stream`, the convolution streams one step higher (so a caller ranks one
 * handle's batches above another's by the priority of the stream it passes first).  When a
 * call repeats an earlier call's pointers, depo counts and event ids, the sequence is recorded
 * as a CUDA graph, and later repeats replay it (up to 8 graphs are kept per handle); the depo
 * values themselves may change between replays.  Results equal those of wct_sim_run_event for
 * each event (up to the float32 summation order of the scatter-add). */
wct_status_t wct_sim_run_batch(wct_sim_t *sim, const wct_depos_t *events, int n_events,
                               float *const *waveforms, void *stream);

/* Per-impact-position responses for one plane: the detector response of §2 step 3 resolved
 * by where the charge sits inside the wire pitch (the transverse grid kept at the patches'
 * impact resolution instead of folded onto wires).  responses: n_phases HOST descriptors, one
 * per impact phase (phase p = sub-bin p of a wire, counted from its low-pitch edge), each
 * [n_wires_resp][n_ticks_resp] with the wire offset k = w - w' (output wire minus the
 * charge's wire) at row k + n_wires_resp / 2; n_phases must equal the plane's
 * n_impact_per_pitch and every phase must share the tick extent of the plane's create-time
 * response (same transform length).  From then on run_event / run_batch / run_host compute
 * that plane as
 *     out[w, t] = sum_{w', p} sum_tau G[n_imp w' + p, t - tau] * R_p[w - w' + kc, tau]
 * (every patch bin added to the phase grid of its sub-bin, every phase grid transformed in one
 * launch, one wire stage summing all phases' stencils, one inverse transform); run_batch runs
 * such events one after the other.  Library memory: n_phases grids of the plane and the
 * spectra of every phase.
 * responses == NULL switches the plane back to the folded mode.  Synchronous. */
wct_status_t wct_sim_set_impact_responses(wct_sim_t *sim, int plane, const wct_response_t *responses, int n_phases);

/* The impact-mode convolution alone: phase_grids DEVICE float32 [n_phases][n_wires][n_ticks]
 * (phase-major), waveform DEVICE [n_wires][n_ticks].  WCT_EINVAL if the plane has no impact
 * responses. */
wct_status_t wct_sim_convolve_impact(wct_sim_t *sim, int plane, const float *phase_grids, float *waveform,
                                     void *stream);

/*
 * One event's depos in HOST memory (same fields and units as wct_depos_t).  Pinned
 * (page-locked) arrays let the uploads overlap device work; pageable arrays work too.
 */
typedef struct {
    const float *t0_us;
    const float *x_mm;
    const float *y_mm;
    const float *z_mm;
    const float *q_e;
    int64_t n;
    uint64_t event_id;
} wct_host_depos_t;

/* The whole DepoTransform (§2) for n_events events from host memory to host memory.
 * events: HOST array of n_events host-depo descriptors; waveforms: HOST array of
 * n_events * n_planes HOST pointers (event-major), each receiving float32 [n_wires][n_ticks]
 * (pinned memory lets the downloads run at full link speed).  Pipelined on three library
 * streams with double-buffered device staging owned by the library (2 x the waveforms of
 * every plane + 2 x the depos of the largest event, counted against the HBM budget): the
 * upload of event e + 1 and the download of event e - 1 overlap the kernels of event e.
 * Synchronous: first waits for all work already enqueued on the device (earlier calls of this
 * handle on any stream share its scratch), returns when every waveform is in host memory, with
 * the status of
 * wct_sim_sync (WCT_EINVAL if invalid depos were skipped).  Results equal those of
 * wct_sim_run_event for each event.  WCT_EINVAL for a NULL or negative argument. */
wct_status_t wct_sim_run_host(wct_sim_t *sim, const wct_host_depos_t *events, int n_events,
                              float *const *waveforms);

/* Digitiser parameters: gain (ADC counts per waveform unit), baseline (counts), noise_rms
 * (counts, white Gaussian), bits (1..15), add_noise (0: no noise). */
typedef struct {
    double gain;
    double baseline;
    double noise_rms;
    int32_t bits;
    int32_t add_noise;
} wct_adc_t;

/* Noise and digitisation, the steps after the convolution of §2: for every bin of a plane's
 * waveform (DEVICE float32 [n_wires][n_ticks]) the ADC code (DEVICE int16, same shape)
 *     code = clamp(floor(gain v + baseline + noise_rms z + 1/2), 0, 2^bits - 1)
 * evaluated in explicitly rounded FP32 in that order (a non-finite value gives 0); z is white
 * Gaussian noise from the Philox stream under the handle's seed, one call per four consecutive
 * ticks of a wire at counter (tick / 4, wire, 0, (0x80 | plane) << 24 | event id), Box-Muller
 * pairs for ticks 4k, 4k+1 and 4k+2, 4k+3.  WCT_EINVAL for bad parameters. */
wct_status_t wct_sim_digitize(wct_sim_t *sim, int plane, const float *waveform, int16_t *adc,
                              const wct_adc_t *params, uint64_t event_id, void *stream);

/* Coloured noise for wct_sim_digitize on one plane: amplitude[f] (HOST, ADC counts) for the
 * n_bins = fft_length / 2 + 1 bins of the plane's transform (wct_sim_plane_info info[3]).
 * While set, the digitiser's noise is, per wire w, the first n_ticks samples of the inverse
 * real DFT of length fft_length (normalised by 1 / fft_length) of
 *     N[w][f] = noise_rms * amplitude[f] * (z_re + i z_im) / sqrt(2)
 * (z_im = 0 at f = 0 and f = fft_length / 2), z from the Philox stream at counter
 * (f / 2, wire, 1, (0x80 | plane) << 24 | event id), words 0,1 for bin 2k and 2,3 for bin 2k+1
 * as Box-Muller pairs; E|N[w][f]|^2 = (noise_rms amplitude[f])^2 for the complex bins.
 * amplitude == NULL switches back to white noise.  Library memory: the spectrum and waveform
 * of one plane.  Synchronous.  WCT_EINVAL for a wrong n_bins or a negative / non-finite
 * amplitude. */
wct_status_t wct_sim_set_noise_spectrum(wct_sim_t *sim, int plane, const float *amplitude, int n_bins);

/* Drift attenuation by the electron lifetime, the step before the rasterization of §2: every
 * depo's charge q becomes the surviving charge of Binomial(q, p), p = exp(-t_d / lifetime),
 * t_d = x / v_drift: its mean q p, or (fluctuate != 0) the normal approximation
 * max(0, q p + sqrt(q p (1 - p)) z) with z drawn from the Philox stream at counter
 * (depo index, 0, 0, 0xFF << 24 | event id) under the seed's key, so every plane sees the same
 * surviving charge.  lifetime_us <= 0 or infinite switches it off (the default).  Applies to
 * every later call of this handle; synchronises the device; drops recorded batch graphs.
 * WCT_EINVAL for a NaN lifetime. */
wct_status_t wct_sim_set_lifetime(wct_sim_t *sim, double lifetime_us, int32_t fluctuate);

/* Synchronise `stream` and return (then clear) the device status word: WCT_OK, or the
 * first device-side error since the last sync (WCT_EINVAL for invalid depos). */
wct_status_t wct_sim_sync(wct_sim_t *sim, void *stream);

/* Per-plane sizes: info[0..8] = {n_wires, n_ticks, fft_length, spectrum_bins,
 * spectrum_row_stride, tile_wires, tile_ticks, n_tiles, spectrum_bins_used}; the last is the
 * response spectrum's support (bins where some response row exceeds 2^-23, FP32 machine
 * epsilon, times the largest magnitude; rounded up to even): the wire stage and inverse transform treat higher bins as zero.
 * Host call, no device work. */
wct_status_t wct_sim_plane_info(const wct_sim_t *sim, int plane, int64_t *info);

/* Stage timing with CUDA events recorded on the caller's stream inside run_event.
 * wct_sim_set_timing(sim, 1) starts (and resets) the record; every following run_event adds
 * one event set per plane.  wct_sim_stage_times waits for the recorded events and writes the
 * mean per run_event call (summed over planes), in microseconds:
 *   us[0] prep + binning, us[1] rasterize + scatter, us[2] forward row FFT,
 *   us[3] wire stage, us[4] inverse row FFT; us[5] (if n > 5) = number of calls timed.
 * While timing, run_batch launches directly (no graph replay) and records, per persistent
 * raster launch, its duration on the raster stream and the span of the convolutions that
 * follow it (the longer of the two convolution streams); with n > 8, us[6] and us[7] receive
 * their sums per run_batch call and us[8] the number of run_batch calls timed. */
wct_status_t wct_sim_set_timing(wct_sim_t *sim, int enable);
wct_status_t wct_sim_stage_times(wct_sim_t *sim, float *us, int n);

/* Counters of this handle: out[0] = kernels launched so far (enqueued directly or recorded
 * into a graph), out[1] = bytes of device memory the library holds, out[2] = batch graphs
 * launched.  Host call, no device work. */
wct_status_t wct_sim_counters(const wct_sim_t *sim, int64_t *out, int n);

/* Failure-detection self-test: launches one kernel whose bounded wait on a shared-memory
 * barrier can never complete (nothing arrives); after limit_cycles SM clocks it gives up and
 * records WCT_ETIMEOUT in the handle's status word, exactly as the library's copy-fed kernels
 * do when a bulk copy never lands.  wct_sim_sync then returns WCT_ETIMEOUT.  The GPU context
 * stays usable.  (The paper has no counterpart.) */
wct_status_t wct_sim_selftest_wait(wct_sim_t *sim, int64_t limit_cycles, void *stream);

/* Human-readable description of the last error on this handle ("" if none). */
const char *wct_sim_last_error(const wct_sim_t *sim);

/* Fault injection for tests of the error paths: after this call the n-th device allocation
 * the library makes (n = 0: the next one), in any handle or in wct_sim_create, fails as if the
 * device were out of memory (WCT_ENOMEM, nothing allocated); later ones succeed again.  n < 0
 * disarms it.  Process-wide, thread-safe; no device work.  Returns WCT_OK. */
wct_status_t wct_debug_fail_alloc(int64_t n);

/* Bounds-checked builds (compiled with -DWCT_BOUNDS_CHECK; a debugging aid standing in for a
 * memory checker): the kernels check the computed indices of the scatter targets, shared-memory
 * boxes, ring slots, tile clears and conversions before use; a violation skips the access,
 * makes the next wct_sim_sync return WCT_EDEVICE and records the first one.  out (HOST int64
 * [3]) receives {source line, index, limit} of that first violation, or zeros.  Synchronous.
 * Returns WCT_OK in a bounds-checked build, WCT_EINVAL in a release build (nothing recorded). */
wct_status_t wct_debug_bounds(wct_sim_t *sim, int64_t *out);

/* The Philox4x32-10 generator the fluctuation uses (Salmon et al., SC'11; §4.1 of the
 * paper), exposed for testing: out[i] = Philox4x32-10(ctr[i], key) for i < n, where ctr
 * and out are DEVICE uint32 [n][4] and key = (seed low word, seed high word). */
wct_status_t wct_philox4x32_10(const uint32_t *ctr, uint64_t seed, int64_t n, uint32_t *out, void *stream);

/*
 * Convolution that allocates no device memory (the paper has no counterpart; this entry
 * point serves callers that may not call cudaMalloc at call time, e.g. code embedded in a
 * host framework that owns every device allocation through its own pool and forbids direct
 * cudaMalloc, or latency-critical paths where the implicit synchronisation of cudaMalloc is
 * not acceptable).
 *
 * Computes the same result as wct_sim_convolve, without a handle: grid and waveform are
 * DEVICE float32 [n_wires][n_ticks] (may be the same buffer); response is a DEVICE float32
 * [n_wires_resp][n_ticks_resp] array in the layout of wct_response_t (odd n_wires_resp <=
 * WCT_MAX_RESPONSE_WIRES).  The response spectrum is recomputed on every call.
 *
 * Scratch: one fixed array of WCT_CONVOLVE_STATIC_SCRATCH_BYTES in device memory, reserved
 * on every GPU that loads the library and held until the process exits.  Sizes whose
 * spectra and tables do not fit in it (roughly 2 * n_wires * (fft_length/2 + 2) * 8 bytes
 * plus the response spectrum and twiddle tables) are rejected with WCT_EINVAL before any
 * launch.  The first call on a device looks up the array's device address and clears its
 * status word (with that device current, synchronously); make that first call before any
 * stream capture.  Every call shares the one array and leaves its contents behind: calls that
 * overlap on the GPU (other streams, other host threads) race with each other and must be
 * serialised by the caller.
 * Device-side errors: the kernels' bounded waits (a bulk copy that never lands) record
 * WCT_ETIMEOUT in a status word at the head of the array instead of aborting; it stays set,
 * across calls, until wct_convolve_static_status reads it.  Returns WCT_OK, WCT_EINVAL
 * (arguments, or too large) or WCT_ECUDA (a launch failed); the launches are asynchronous, so
 * WCT_OK means "enqueued": read wct_convolve_static_status before trusting the waveform.
 */
#define WCT_CONVOLVE_STATIC_SCRATCH_BYTES (16u << 20)
wct_status_t wct_convolve_static(const float *grid, int32_t n_wires, int32_t n_ticks, const float *response,
                                 int32_t n_wires_resp, int32_t n_ticks_resp, float *waveform, void *stream);

/* Status of the wct_convolve_static calls on the current device since the last read:
 * synchronises `stream` (the stream of those calls), then returns and clears the status word
 * of the fixed array: WCT_OK, WCT_ETIMEOUT (a bounded wait gave up: that call's waveform is
 * incomplete) or WCT_EDEVICE; WCT_ECUDA if the synchronisation or the read failed.  Allocates
 * nothing.  (The paper has no counterpart.) */
wct_status_t wct_convolve_static_status(void *stream);

/* Self-test of that error path: one kernel whose bounded wait on a shared-memory barrier can
 * never complete gives up after limit_cycles SM clocks and records WCT_ETIMEOUT in the fixed
 * array's status word, as the convolution's copy-fed kernels do when a bulk copy never lands;
 * wct_convolve_static_status then returns WCT_ETIMEOUT and the context stays usable.
 * Allocates nothing.  (The paper has no counterpart.) */
wct_status_t wct_convolve_static_selftest_wait(int64_t limit_cycles, void *stream);

/*
 * A field response (input of the detector response of §2 step 3, which the paper takes as
 * given): the current induced on ONE wire by a unit charge drifting along each of n_paths
 * paths, the paths at charge positions path_pos_mm[j] across the pitch direction relative to
 * that wire's centre (strictly increasing), every path sampled n_samples times at period_us
 * from one common time origin: current[j][s], in unit charges per microsecond.  This is the
 * form a field calculation produces (currents on a fine time grid for drift paths at
 * sub-pitch spacing).  If every position is >= 0 the field is taken as mirror-symmetric,
 * I(-x) = I(x).  Between paths the current is interpolated linearly in x; beyond the
 * outermost path it is zero.  All HOST memory, read only during the call.
 */
typedef struct {
    int32_t n_paths;            /* >= 2 */
    int32_t n_samples;          /* >= 1 */
    double period_us;           /* > 0 */
    const double *path_pos_mm;  /* [n_paths] */
    const double *current;      /* [n_paths][n_samples] */
} wct_field_response_t;

/*
 * The tick-sampled detector response from a field response and an electronics impulse
 * response electronics[0 .. n_elec) sampled at the same period (e.g. a CR-RC^2 shaper times
 * its gain):
 *     R_p[r][tau] = period * sum_s I(y_p - (r - K) pitch, s period) * E[tau m - s],
 * the field current convolved with the electronics in time and sampled at the tick times
 * (m = tick_us / period_us must be an integer), for the wire at offset r - K from the wire
 * the charge is on (K = n_wires_resp / 2, n_wires_resp odd) and the charge at the centre of
 * impact sub-bin p of its wire, y_p = ((p + 1/2) / n_impact - 1/2) pitch.
 *   impact_out  HOST float [n_impact][n_wires_resp][n_ticks_resp] or NULL: the per-impact-
 *               position responses (wct_sim_set_impact_responses, one per phase);
 *   folded_out  HOST float [n_wires_resp][n_ticks_resp] or NULL: their average over the
 *               n_impact phases, the response of a charge spread evenly across the pitch
 *               (wct_sim_create's response for the folded mode).
 * Host computation in FP64, no device work, no handle.  Returns WCT_OK or WCT_EINVAL (sizes,
 * positions not strictly increasing, a tick that is not a whole number of periods, a
 * non-finite value).
 */
wct_status_t wct_response_from_field(const wct_field_response_t *field, const double *electronics, int32_t n_elec,
                                     double pitch_mm, int32_t n_impact, double tick_us, int32_t n_wires_resp,
                                     int32_t n_ticks_resp, float *impact_out, float *folded_out);

#ifdef __cplusplus
}
#endif
#endif /* WCT_SIM_H */
