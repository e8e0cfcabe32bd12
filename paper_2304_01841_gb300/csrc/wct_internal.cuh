// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wct_sim.h"

namespace wct {

// ------------------------------------------------------------------------------------------
// Per-depo descriptor produced by the prep kernel (32 bytes, two float4 loads).
//   mu_t / mu_p : centre relative to the window's first bin, in bin units (FP64 -> FP32)
//   inv_t/inv_p : 1 / (sqrt(2) sigma) in 1/bin, 0 for a point charge
//   lo_t / lo_p : first window bin (absolute tick / impact bin)
//   nt / np     : window extent; nt == 0 marks an invalid or empty depo
// ------------------------------------------------------------------------------------------
struct __align__(16) DepoDesc {
    float mu_t, mu_p, inv_t, inv_p;
    float q;
    int32_t lo_t, lo_p;
    int16_t nt, np;
};
static_assert(sizeof(DepoDesc) == 32, "DepoDesc must stay 32 bytes");

// Geometry / physics constants of one plane, FP64 where the window is decided.
struct PlaneParams {
    double pitch, origin, cos_a, sin_a, tick, tw0, dp;   // dp = pitch / n_imp
    double DL, DT, v, nsigma;                            // DL, DT in mm^2/us
    double inv_tick, inv_vtick, inv_dp;                  // 1/tick, 1/(v tick), 1/dp
    // the same constants as double-floats (hi, lo): inv_vtick, inv_tick, tw0, cos_a, sin_a,
    // origin, inv_dp; the window's fast path runs on them in FP32
    float ff[7][2];
    float kt, kp;                                        // sigma_t = kt sqrt(x), sigma_p = kp sqrt(x)
    // drift attenuation: q -> q exp(-x / (v lifetime)) (0: none), optionally fluctuated
    float inv_v_lifetime;                                // 1 / (v lifetime) in 1/mm
    int32_t fluct_absorb;
    int32_t n_imp, n_wires, n_ticks, plane_index;
    int32_t fluctuate;
    uint32_t key0, key1;
    uint32_t rk[20];                                     // Philox round keys of (key0, key1)
    int32_t tile_w, tile_t, n_tiles_w, n_tiles_t;
    int32_t raster_schedule;                             // 0 warp-level chunks, 1 CTA-level chunks
};

// Device status word codes (same values as wct_status_t).
enum : int32_t { ST_OK = 0, ST_EINVAL = 1, ST_ETIMEOUT = 4, ST_EDEVICE = 6 };

// Radix plan of a complex FFT of length M = fft_length / 2 (Stockham, radices 2..8).
struct FFTPlan {
    int32_t M;            // complex length
    int32_t n_stages;
    int32_t radix[12];
    uint64_t radix_code;  // radix[s] in bits [4s, 4s+4): read in registers, no local-memory array
    int32_t fft_len;      // real length P = 2M
    int32_t F;            // spectrum bins = M + 1
    int32_t Fs;           // spectrum row stride (complex elements), even
    int32_t Fu;           // spectrum bins carried through the wire stage (even, <= Fs): the
                          // response spectrum's support; bins above it are treated as zero
    float2 *tw;           // device: exp(-2 pi i k / M), k < M
    float2 *rtw;          // device: exp(-2 pi i k / P), k <= M
    int32_t row_schedule; // row kernels: 0 register-staged, 1 one persistent CTA per SM,
                          // 2 two paired CTAs per SM, 3 paired with composite radices
};

// One (event, plane) pair of a batched rasterize + scatter launch.
struct BatchItem {
    const float *t0, *x, *y, *z, *q;
    int64_t n;
    float *grid;
    unsigned long long *grid64;   // deterministic mode: fixed-point grid the raster adds to
    uint32_t *flags;       // touched-tile flags of grid (or null)
    int64_t chunk_begin;   // first CTA of this pair (prefix sum of its chunk counts)
    uint32_t event_lo;
    int32_t plane;
};

// Passed by value as the kernel parameter (up to kBatchItems pairs, ~21 KB).
constexpr int kBatchItems = 256;
constexpr int kMaxPlanesDev = 8;
struct BatchTable {
    PlaneParams plane[kMaxPlanesDev];
    BatchItem item[kBatchItems];
    int32_t n_items;
};

// ---- launchers (stream-ordered; return cudaError_t of the launch) -------------------------
cudaError_t launch_prep(const wct_depos_t &d, const PlaneParams &pp, DepoDesc *desc, int32_t *tile_count,
                        int64_t *patch_size, int32_t *status, cudaStream_t s);
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);

// Deterministic mode (wct_opts_t::deterministic): the rasterizers add fixed-point values,
// round(v * kFixScale), to a 64-bit integer grid (grid64 / BatchItem::grid64) instead of floats
// to `grid`; launch_fix_tiles then adds the listed tiles to the float grid and zeroes them.
constexpr float kFixScale = 1048576.f;   // 2^20 units per electron
cudaError_t launch_raster_chunks(const wct_depos_t &d, const PlaneParams &pp, uint32_t event_lo, float *grid,
                                 int32_t *status, cudaStream_t s, uint32_t *flags = nullptr,
                                 unsigned long long *grid64 = nullptr);
cudaError_t launch_raster_batch(const BatchTable &tab, int64_t total_chunks, int32_t *status, cudaStream_t s,
                                bool det = false);
// One persistent launch over every warp-chunk of the table's pairs (total_chunks warp-chunks of
// 8 depos, chunk_begin in warp-chunks): the warps take chunks from *counter (reset on `s`
// first) until none is left.
cudaError_t launch_raster_batch_persistent(const BatchTable &tab, int64_t total_chunks, unsigned long long *counter,
                                           int32_t *status, cudaStream_t s, bool det);
// grid[r][c] += g64[r][c] / kFixScale and g64[r][c] = 0 over the tiles listed in flags (the
// flag layout below, for an n_rows x n_cols grid with tile_w x tile_t tiles; flags only read)
cudaError_t launch_fix_tiles(const uint32_t *flags, int n_rows, int n_cols, int tile_w, int tile_t,
                             unsigned long long *g64, float *grid, cudaStream_t s, int32_t *status = nullptr);
// Touched-tile flags: the fused rasterizers set flags[tile] = 1 for every tile (tile_w wires x
// tile_t ticks, pp's tiling) that a depo's window overlaps and list each such tile once
// (flags: n_tiles flags, a count, a done-counter, the list; tile_flag_words(pp) words, all
// zero initially).  Clearing zeroes the listed tiles of the grid and resets the flags and
// the list, restoring an all-zero grid: a side job of the wire stage (ClearJob).
size_t tile_flag_words(const PlaneParams &pp);

struct ClearJob {
    float *grid = nullptr;        // null: no job
    uint32_t *flags = nullptr;
    int n_wires = 0, n_ticks = 0, tile_w = 0, tile_t = 0, n_tiles_t = 0, n_tiles = 0;
};
ClearJob clear_job(float *grid, uint32_t *flags, const PlaneParams &pp);

// The listed tiles of job.grid, CTA `cta` of `n_ctas` taking list entries cta, cta + n_ctas,
// ...; threads 0 .. threads - 1 (a multiple of 32) take part and meet at named barrier 1.
// Every CTA of the launch must call it exactly once: thread 0 reads the count for its CTA,
// and the last CTA to have read it resets the count and the done-counter.
__device__ __forceinline__ void clear_listed_tiles(const ClearJob &job, unsigned cta, unsigned n_ctas, int threads) {
    __shared__ uint32_t s_count;
    const int tid = threadIdx.x;
    if (tid >= threads) return;
    uint32_t *flags = job.flags;
    const int n_tiles = job.n_tiles;
    if (tid == 0) {
        s_count = min(*(volatile uint32_t *)&flags[n_tiles], (uint32_t)n_tiles);
        if (atomicAdd(&flags[n_tiles + 1], 1u) == n_ctas - 1) {   // every CTA has read the count
            flags[n_tiles] = 0u;
            flags[n_tiles + 1] = 0u;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
    const uint32_t count = s_count;
    const int warp = tid >> 5, lane = tid & 31, n_warps = threads >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(job.grid) & 15) == 0 && (job.n_ticks & 3) == 0 && (job.tile_t & 3) == 0;
    for (uint32_t i = cta; i < count; i += n_ctas) {
        const int t = (int)flags[n_tiles + 2 + i];
        if (t < 0 || t >= n_tiles) continue;
        const int tw = t / job.n_tiles_t, tt = t - tw * job.n_tiles_t;
        const int w0 = tw * job.tile_w, w1 = min(w0 + job.tile_w, job.n_wires);
        const int c0 = tt * job.tile_t, width = min(job.tile_t, job.n_ticks - c0);
        if (vec && (width & 3) == 0) {
            for (int w = w0 + warp; w < w1; w += n_warps) {
                float4 *row = reinterpret_cast<float4 *>(job.grid + (size_t)w * job.n_ticks + c0);
                for (int c = lane; c < (width >> 2); c += 32) row[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int w = w0 + warp; w < w1; w += n_warps)
                for (int c = lane; c < width; c += 32) job.grid[(size_t)w * job.n_ticks + c0 + c] = 0.f;
        }
        if (tid == 0) flags[t] = 0u;
    }
}
int64_t raster_chunk_count(int64_t n, int schedule);
cudaError_t launch_rasterize_patches(int64_t n, const DepoDesc *desc, const int64_t *offsets, const PlaneParams &pp,
                                     uint32_t event_lo, float *patches, int64_t *patch_desc, cudaStream_t s,
                                     int64_t slot = 0);
// offsets == nullptr: depo i's patch at i * slot (the scan-free slots)
cudaError_t launch_fit_slots(int64_t n, DepoDesc *desc, int64_t slot, int32_t *status, cudaStream_t s);
cudaError_t launch_bin_patches(int64_t n, const int64_t *patch_desc, const PlaneParams &pp, int32_t *tile_count,
                               int32_t *status, cudaStream_t s);
cudaError_t launch_fill_patches(int64_t n, const int64_t *patch_desc, const PlaneParams &pp, const int32_t *tile_off,
                                int32_t *tile_cursor, int32_t *tile_list, int64_t list_cap, int32_t *status,
                                cudaStream_t s);
cudaError_t launch_tile_scatter_patches(const int64_t *patch_desc, const float *patches, const int32_t *tile_off,
                                        const int32_t *tile_list, int64_t list_cap, const PlaneParams &pp, float *grid,
                                        cudaStream_t s, bool det = false, int32_t *status = nullptr);

// act (optional, n_rows bytes): rows with act[row] == 0 are all zero; the paired kernels skip
// them (their spectra rows are left unwritten and must be read as zero, as the wire stage does
// when given the same act); other kernels transform every row
cudaError_t launch_row_r2c(const FFTPlan &p, const float *in, int64_t in_stride, int n_in_cols, int n_rows,
                           float2 *spec, cudaStream_t s, int32_t *status = nullptr, const uint8_t *act = nullptr);
// accumulate: out += the stencil instead of out = (the per-phase sum of the impact mode)
// act (optional, [n_phases][n_wires]): spectrum rows with act == 0 are read as zero
cudaError_t launch_wire_stage(const FFTPlan &p, const float2 *spec, const float2 *resp_spec, int n_wires,
                              float2 *out, cudaStream_t s, int32_t *status = nullptr, const ClearJob *clear = nullptr,
                              bool accumulate = false, int n_phases = 1, const uint8_t *act = nullptr);
// act_s [n_phases][n_wires] / act_t [n_wires] of a library grid (the phase grids stacked, in the
// impact mode) from its touched-tile flags (see k_row_activity)
cudaError_t launch_row_activity(const uint32_t *flags, int n_tiles_t, int tile_w, int n_wires, uint8_t *act_s,
                                uint8_t *act_t, cudaStream_t s, int n_phases = 1);
// n_phases > 1 (impact mode): spec holds n_phases spectra [phase][wire][Fs] and resp_spec
// n_phases response spectra [phase][21][Fs]; out = (out +) the sum over phases of their stencils
// Noise + digitisation: code = clamp(floor(gain v + baseline + noise_rms z + 1/2), 0, max_code)
struct AdcParams {
    float gain, baseline, noise_rms, max_code;
    int32_t add_noise;
    uint32_t rk[20];            // Philox round keys of the seed
    const float *noise_wave;    // coloured noise [n_wires][n_ticks] to add (null: white noise)
};
// Coloured-noise spectrum [n_wires][Fs] (scale folds the inverse transform's 1/M and noise_rms)
cudaError_t launch_noise_spectrum(const float *amp, int F, int M, int n_wires, int Fs, float scale, const AdcParams &a,
                                  uint32_t c3, float2 *spec, cudaStream_t s);
cudaError_t launch_digitize(const float *wf, int16_t *adc, int n_wires, int n_ticks, const AdcParams &a, uint32_t c3,
                            cudaStream_t s);
// Impact mode, fused: patches of the depos (windows from launch_prep) added bin by bin to the
// n_imp phase grids [phase][wire][tick], no patch buffer.
// flags: touched-tile flags of the phase grids seen as one (n_imp * n_wires) x n_ticks grid
// with pp's tiling (or null)
cudaError_t launch_raster_phases(int64_t n, const DepoDesc *desc, const PlaneParams &pp, uint32_t event_lo,
                                 float *grids, uint32_t *flags, cudaStream_t s, unsigned long long *grids64 = nullptr,
                                 int32_t *status = nullptr);

// act (optional): output rows with act[row] == 0 are zero; the paired kernels write them as zeros
// without a transform (their spectrum rows need not exist), other kernels transform every row
cudaError_t launch_row_c2r(const FFTPlan &p, const float2 *spec, int n_rows, float *out, int64_t out_stride,
                           int n_out_cols, cudaStream_t s, int32_t *status = nullptr, const uint8_t *act = nullptr);
cudaError_t launch_scale_spectrum(float2 *spec, int64_t n, float scale, cudaStream_t s);
cudaError_t launch_make_twiddles(const FFTPlan &p, cudaStream_t s);
cudaError_t launch_wait_selftest(long long limit, int32_t *status, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t *out, cudaStream_t s);

}  // namespace wct
