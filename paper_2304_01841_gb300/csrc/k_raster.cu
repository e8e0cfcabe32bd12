// Rasterization (+ fluctuation) and scatter-add (paper §2, steps 1 and 2).
//
// Fused path, k_raster_chunks (below): depo-parallel, the patch of each depo is evaluated
// folded onto wires (the sum over a wire's impact sub-bins of the fluctuated bin charges),
// accumulated in shared memory per chunk of depos and then added to the grid.  The paper's
// scatter-add adds every patch bin with a global atomic (§2, §5.2); here a chunk of track
// depos shares one shared-memory box, so the global adds shrink to one per touched bin.
//
// The fluctuation renormalises each patch to its charge over the depo's whole window.
// Because rescaling is linear, the fold is taken on the unscaled fluctuated charges and the
// scale q / sum is applied afterwards.
//
// Unfused path: k_rasterize_patches (one warp per depo) writes every depo's full patch;
// k_tile_scatter_patches sums caller-supplied patches per output tile in shared memory and
// writes each tile once.
#include <algorithm>
#include <climits>
#include <mutex>

#include "wct_internal.cuh"
#include "wct_device.cuh"

namespace wct {

namespace {

// Accumulation into a grid or a shared-memory box.  Deterministic mode (wct_opts_t::
// deterministic): each contribution is rounded to fixed point (kFixScale units per electron)
// and summed as a 64-bit integer; integer addition is associative, so the sums do not depend
// on the order in which the atomics land (warp scheduling, batching, depo order).
template <bool DET>
struct Acc;
template <>
struct Acc<false> {
    using T = float;
    __device__ __forceinline__ static void add(float *p, float v) { atomicAdd(p, v); }
};
template <>
struct Acc<true> {
    using T = unsigned long long;
    __device__ __forceinline__ static void add(unsigned long long *p, float v) {
        atomicAdd(p, (unsigned long long)__float2ll_rn(v * kFixScale));   // two's complement sum
    }
};

constexpr int kTileWarps = 8;
constexpr int kWT = WCT_MAX_WINDOW_TICKS + 1;                 // per-warp time weights (+1 edge)
constexpr int kWBuf = kWT + WCT_MAX_WINDOW_IMPACTS + 1;       // per-warp weight buffer (floats)

// Warp-cooperative 1D weights of one axis: w[i] = (erf(x_{i+1}) - erf(x_i)) / 2 with
// x_i = (i - mu) * inv (window-relative bin edges), normalised to sum 1.  inv == 0 marks a
// point charge (single bin of weight 1).  `w` has room for n + 1 entries.
__device__ __forceinline__ void axis_weights(float *w, int n, float mu, float inv, int lane) {
    if (inv == 0.f) {
        if (lane == 0) w[0] = 1.f;
        __syncwarp();
        return;
    }
    for (int i = lane; i <= n; i += 32) w[i] = erff(((float)i - mu) * inv);
    __syncwarp();
    float part = 0.f;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        float v = 0.f;
        if (i < n) v = 0.5f * (w[i + 1] - w[i]);
        __syncwarp();
        if (i < n) w[i] = v;
        part += v;
        __syncwarp();
    }
    const float inv_sum = 1.f / warp_sum(part);
    for (int i = lane; i < n; i += 32) w[i] *= inv_sum;
    __syncwarp();
}

// One (tick, wire) item of a depo's window folded onto wires.
struct Item {
    int a;          // window-relative tick
    int tick;       // absolute tick
    int wire;       // absolute wire
    int sub_lo;     // first sub-bin of the wire inside the window
    int sub_hi;     // one past the last
    int j_base;     // window-relative impact index of sub-bin 0 of this wire
};

__device__ __forceinline__ Item make_item(int it, int nw, int wl, const DepoDesc &d, int n_imp) {
    Item f;
    // it / nw without an integer division: the quotient (it + 1/2) / nw is at most 128 and at
    // least 1/(2 nw) >= 1e-3 away from an integer, far beyond the ~3e-5 error of the SFU divide
    f.a = (int)__fdividef((float)it + 0.5f, (float)nw);
    f.wire = wl + (it - f.a * nw);
    f.tick = d.lo_t + f.a;
    const int first = f.wire * n_imp;                     // absolute impact of sub-bin 0
    f.j_base = first - d.lo_p;
    f.sub_lo = max(first, d.lo_p) - first;
    f.sub_hi = min(first + n_imp, d.lo_p + (int)d.np) - first;
    return f;
}

__device__ __forceinline__ float fold_plain(const Item &f, const float *wt, const float *wp, float q) {
    float s = 0.f;
    for (int sub = f.sub_lo; sub < f.sub_hi; ++sub) s += wp[f.j_base + sub];
    return q * wt[f.a] * s;
}

// Fluctuated, not yet rescaled, folded charge of one item: the sum over the wire's sub-bins
// in the window of max(0, q w + sqrt(q w (1 - w)) z), w = w_t * w_p (the variance m - m w
// with m = q w as one fused multiply-add: one rounding, never negative).  z comes from the
// counter-based pool: Philox4x32-10 of (depo, tick, wire * G + group, c3) under the key;
// a call serves a group of four sub-bins, lanes 0/1 from the Box-Muller pair of words 0/1
// and lanes 2/3 from words 2/3.
__device__ __forceinline__ float fold_fluct(const Item &f, const float *wt, const float *wp, float q, uint32_t depo,
                                            const PlaneParams &pp, uint32_t c3, const uint32_t (&rk)[20]) {
    const int G = (pp.n_imp + 3) >> 2;
    const float wa = wt[f.a];
    float acc = 0.f;
    const int g0 = f.sub_lo >> 2, g1 = (f.sub_hi - 1) >> 2;
    for (int g = g0; g <= g1; ++g) {
        const uint4 x = philox4x32_10_rk(make_uint4(depo, (uint32_t)f.tick, (uint32_t)(f.wire * G + g), c3), rk);
        const int sb = g << 2;
        const int l0 = max(f.sub_lo - sb, 0), l1 = min(f.sub_hi - sb, 4);   // lanes [l0, l1)
        float z[4];
        if (l0 < 2) {
            const float2 p = box_muller(x.x, x.y);
            z[0] = p.x;
            z[1] = p.y;
        }
        if (l1 > 2) {
            const float2 p = box_muller(x.z, x.w);
            z[2] = p.x;
            z[3] = p.y;
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (l >= l0 && l < l1) {
                const float w = wa * wp[f.j_base + sb + l];
                const float m = q * w;
                const float v = fmaf(sfu_sqrt(fmaf(-m, w, m)), z[l], m);
                acc += fmaxf(v, 0.f);
            }
        }
    }
    return acc;
}

// Flag the tiles (tile_w rows x tile_t ticks of a grid with n_tiles_t tiles per row band)
// covering rows [r0, r1] x ticks [b0, b1], listing each newly flagged tile (layout below).
__device__ __forceinline__ void flag_tiles(uint32_t *flags, int n_tiles, int n_tiles_t, int tile_w, int tile_t, int r0,
                                           int r1, int b0, int b1) {
    for (int tw = r0 / tile_w; tw <= r1 / tile_w; ++tw)
        for (int tt = b0 / tile_t; tt <= b1 / tile_t; ++tt) {
            const int t = tw * n_tiles_t + tt;
            if (flags[t] == 0u && atomicExch(&flags[t], 1u) == 0u) {
                const uint32_t slot = atomicAdd(&flags[n_tiles], 1u);
                flags[n_tiles + 2 + slot] = (uint32_t)t;
            }
        }
}

// Flag the grid tiles that depo d's window overlaps (clamped to the grid).  flags holds
// n_tiles flags, then a counter and a done-counter, then the list of flagged tiles: the
// first depo to flag a tile appends it to the list.
__device__ __forceinline__ void mark_tiles(uint32_t *flags, const PlaneParams &pp, const DepoDesc &d, int wl, int nw) {
    if (!flags || d.nt == 0) return;
    const int a0 = max(wl, 0), a1 = min(wl + nw - 1, pp.n_wires - 1);
    const int b0 = max(d.lo_t, 0), b1 = min(d.lo_t + (int)d.nt - 1, pp.n_ticks - 1);
    if (a0 > a1 || b0 > b1) return;
    flag_tiles(flags, pp.n_tiles_w * pp.n_tiles_t, pp.n_tiles_t, pp.tile_w, pp.tile_t, a0, a1, b0, b1);
}

__device__ __forceinline__ uint32_t counter_c3(const PlaneParams &pp, uint32_t event_lo) {
    return ((uint32_t)pp.plane_index << 24) | (event_lo & 0xFFFFFFu);
}

// ------------------------------------------------------------------------------------------
// Fused rasterize + fluctuate + fold + scatter, balanced over depos.
//
// One CTA takes a chunk of kChunk consecutive depos (consecutive depos of a track are close
// in space).  Its threads (1) compute every depo's FP64 window, (2) compute all erf bin
// weights of the chunk, flattened over (depo, bin), (3) evaluate all (tick, wire) items of
// the chunk, flattened over (depo, item) so every lane has work, summing each depo's
// fluctuated charge with a segmented warp reduction, (4) add the rescaled items into a
// shared-memory box covering the chunk's footprint on the grid, and (5) add the box to the
// grid in global memory, one atomic per touched bin.  A chunk whose footprint does not fit
// the box (scattered depos) adds its items to global memory directly.  The grid is zeroed
// before the launch.
// ------------------------------------------------------------------------------------------
constexpr int kChunkThreads = 256;
constexpr int kChunk = 64;
constexpr int kItemCap = 6144;     // items cached per pass (a wider single depo is recomputed)
constexpr int kWCap = 2048;        // >= 128 + 512, the weights of the largest window
constexpr int kBoxCap = 6144;      // wires x ticks accumulated in shared memory

struct ChunkSmem {
    DepoDesc d[kChunk];
    int item_off[kChunk + 1];
    int w_off[kChunk + 1];
    int wl[kChunk];
    int nw[kChunk];
    float nrm_t[kChunk];
    float nrm_p[kChunk];
    float sum[kChunk];
    int pass_end;
    int use_box, box_w0, box_t0, box_nw, box_nt;
    float w[kWCap];
    float val[kItemCap];
    float box[kBoxCap];
    uint8_t slot[kItemCap];   // depo of each cached item (chunk-relative)
};

// largest j in [lo, hi) with off[j] <= k (off non-decreasing, off[lo] <= k)
__device__ __forceinline__ int find_slot(const int *off, int lo, int hi, int k) {
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Segmented warp sum over lanes with equal (sorted) keys; the last lane of each segment adds
// the segment's total to sums[key].  Keys < 0 are ignored.
__device__ __forceinline__ void segmented_add(int key, float v, float *sums) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float vv = __shfl_up_sync(0xffffffffu, v, o);
        const int kk = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && kk == key) v += vv;
    }
    const int next = __shfl_down_sync(0xffffffffu, key, 1);
    if (key >= 0 && (lane == 31 || next != key)) atomicAdd(&sums[key], v);
}

// One chunk of one event's depos for one plane (the body of the fused kernels below).
__device__ __forceinline__ void raster_chunk(ChunkSmem &S, const float *__restrict__ t0, const float *__restrict__ x,
                                             const float *__restrict__ y, const float *__restrict__ z,
                                             const float *__restrict__ q, int64_t n, const PlaneParams &pp,
                                             uint32_t event_lo, float *__restrict__ grid, int32_t *status,
                                             int64_t chunk, const uint32_t (&RK)[20], uint32_t *flags) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t c0 = chunk * kChunk;
    const int cn = (int)((n - c0) < kChunk ? (n - c0) : kChunk);
    const uint32_t c3 = counter_c3(pp, event_lo);

    if (tid < cn) {
        const int64_t i = c0 + tid;
        DepoDesc d;
        if (!depo_window(t0[i], x[i], y[i], z[i], q[i], pp, d)) set_status(status, ST_EINVAL);
        else d.q = drift_absorb(d.q, x[i], (uint32_t)i, event_lo, pp);
        S.d[tid] = d;
        int wl = 0, nw = 0;
        if (d.nt > 0) {
            wl = floor_div(d.lo_p, pp.n_imp);
            nw = floor_div(d.lo_p + d.np - 1, pp.n_imp) - wl + 1;
        }
        S.wl[tid] = wl;
        S.nw[tid] = nw;
        mark_tiles(flags, pp, d, wl, nw);
        // sum of a window's unnormalised weights telescopes to (erf(x_n) - erf(x_0)) / 2
        S.nrm_t[tid] = d.inv_t == 0.f ? 1.f : 1.f / (erff(((float)d.nt - d.mu_t) * d.inv_t) - erff(-d.mu_t * d.inv_t));
        S.nrm_p[tid] = d.inv_p == 0.f ? 1.f : 1.f / (erff(((float)d.np - d.mu_p) * d.inv_p) - erff(-d.mu_p * d.inv_p));
        S.sum[tid] = 0.f;
    }
    __syncthreads();

    for (int s = 0; s < cn;) {
        if (tid == 0) {
            // pack depos [s, e) whose items and weights fit, and bound their footprint
            int it = 0, ww = 0, e = s;
            int w0 = INT_MAX, w1 = INT_MIN, t0b = INT_MAX, t1b = INT_MIN;
            for (; e < cn; ++e) {
                const DepoDesc &d = S.d[e];
                const int ni = (int)d.nt * S.nw[e], nwt = (int)d.nt + (int)d.np;
                if (e > s && (it + ni > kItemCap || ww + nwt > kWCap)) break;
                S.item_off[e] = it;
                S.w_off[e] = ww;
                it += ni;
                ww += nwt;
                if (d.nt > 0) {
                    const int a0 = max(S.wl[e], 0), a1 = min(S.wl[e] + S.nw[e] - 1, pp.n_wires - 1);
                    const int b0 = max(d.lo_t, 0), b1 = min(d.lo_t + (int)d.nt - 1, pp.n_ticks - 1);
                    if (a0 <= a1 && b0 <= b1) {
                        w0 = min(w0, a0); w1 = max(w1, a1);
                        t0b = min(t0b, b0); t1b = max(t1b, b1);
                    }
                }
            }
            S.item_off[e] = it;
            S.w_off[e] = ww;
            S.pass_end = e;
            const bool any = w0 <= w1;
            const int64_t area = any ? (int64_t)(w1 - w0 + 1) * (t1b - t0b + 1) : 0;
            S.use_box = any && area <= kBoxCap;
            S.box_w0 = w0;
            S.box_t0 = t0b;
            S.box_nw = any ? w1 - w0 + 1 : 0;
            S.box_nt = any ? t1b - t0b + 1 : 0;
        }
        __syncthreads();
        const int e = S.pass_end;
        const int n_items = S.item_off[e] - S.item_off[s];
        const int i_base = S.item_off[s];
        const int n_w = S.w_off[e] - S.w_off[s];
        const int w_base = S.w_off[s];
        const bool use_box = S.use_box;
        const int bnt = S.box_nt, bw0 = S.box_w0, bt0 = S.box_t0;
        if (use_box)
            for (int k = tid; k < S.box_nw * bnt; k += kChunkThreads) S.box[k] = 0.f;
        // (2) bin weights, flattened over (depo, bin): w = (erf(x_{i+1}) - erf(x_i)) * nrm
        for (int k = tid; k < n_w; k += kChunkThreads) {
            const int j = find_slot(S.w_off, s, e, w_base + k);
            const DepoDesc &d = S.d[j];
            const int r = w_base + k - S.w_off[j];
            float w;
            if (r < d.nt) {
                w = d.inv_t == 0.f ? 1.f
                                   : (erff(((float)(r + 1) - d.mu_t) * d.inv_t) - erff(((float)r - d.mu_t) * d.inv_t)) *
                                         S.nrm_t[j];
            } else {
                const int rr = r - d.nt;
                w = d.inv_p == 0.f ? 1.f
                                   : (erff(((float)(rr + 1) - d.mu_p) * d.inv_p) - erff(((float)rr - d.mu_p) * d.inv_p)) *
                                         S.nrm_p[j];
            }
            S.w[k] = w;
        }
        __syncthreads();
        // (3) items, flattened over (depo, item)
        for (int base = tid - lane; base < n_items; base += kChunkThreads) {
            const int k = base + lane;
            int j = -1;
            float v = 0.f;
            if (k < n_items) {
                j = find_slot(S.item_off, s, e, i_base + k);
                const DepoDesc &d = S.d[j];
                const Item f = make_item(i_base + k - S.item_off[j], S.nw[j], S.wl[j], d, pp.n_imp);
                const float *wt = S.w + (S.w_off[j] - w_base);
                const float *wp = wt + d.nt;
                v = pp.fluctuate ? fold_fluct(f, wt, wp, d.q, (uint32_t)(c0 + j), pp, c3, RK) : fold_plain(f, wt, wp, d.q);
                if (k < kItemCap) {   // a single very wide depo may exceed the cache
                    S.val[k] = v;
                    S.slot[k] = (uint8_t)j;
                }
            }
            if (pp.fluctuate) segmented_add(j, v, S.sum);
        }
        __syncthreads();
        // (4) rescale and accumulate (box in shared memory, or the grid directly)
        for (int k = tid; k < n_items; k += kChunkThreads) {
            const int j = k < kItemCap ? (int)S.slot[k] : find_slot(S.item_off, s, e, i_base + k);
            const DepoDesc &d = S.d[j];
            const Item f = make_item(i_base + k - S.item_off[j], S.nw[j], S.wl[j], d, pp.n_imp);
            if (f.wire < 0 || f.wire >= pp.n_wires || f.tick < 0 || f.tick >= pp.n_ticks) continue;
            const float *wt = S.w + (S.w_off[j] - w_base);
            float v;
            if (k < kItemCap) v = S.val[k];
            else v = pp.fluctuate ? fold_fluct(f, wt, wt + d.nt, d.q, (uint32_t)(c0 + j), pp, c3, RK)
                                  : fold_plain(f, wt, wt + d.nt, d.q);
            if (pp.fluctuate) {
                const float sm = S.sum[j];
                if (sm > 0.f) v *= d.q / sm;
                else v = fold_plain(f, wt, wt + d.nt, d.q);
            }
            if (use_box) atomicAdd(&S.box[(f.wire - bw0) * bnt + (f.tick - bt0)], v);
            else atomicAdd(&grid[(int64_t)f.wire * pp.n_ticks + f.tick], v);
        }
        __syncthreads();
        // (5) the box's touched bins to the grid
        if (use_box) {
            const int area = S.box_nw * bnt;
            for (int k = tid; k < area; k += kChunkThreads) {
                const float v = S.box[k];
                if (v != 0.f) {
                    const int r = k / bnt;
                    atomicAdd(&grid[(int64_t)(bw0 + r) * pp.n_ticks + bt0 + (k - r * bnt)], v);
                }
            }
        }
        __syncthreads();
        s = e;
    }
}

// ------------------------------------------------------------------------------------------
// Warp-level variant: each warp owns kWarpDepos consecutive depos and runs the same steps with
// warp-synchronous code only (no CTA barriers, so a warp never waits for a slower one), with
// its own weights / item cache / accumulation box in shared memory.
// ------------------------------------------------------------------------------------------
constexpr int kWarpDepos = 8;
constexpr int kWarpsPerCta = 4;
constexpr int kWItemCap = 384;
constexpr int kWWCap = 648;        // >= 129 + 513, the bin edges of the largest window
constexpr int kWBoxCap = 304;

template <bool DET>
struct WarpSmem {
    DepoDesc d[kWarpDepos];
    int item_off[kWarpDepos + 1];
    int w_off[kWarpDepos + 1];
    int wl[kWarpDepos];
    int nw[kWarpDepos];
    float nrm_t[kWarpDepos];
    float nrm_p[kWarpDepos];
    float sum[kWarpDepos];     // fluctuated sum of each depo's items, then its rescale q / sum
    int pass_end, use_box, box_w0, box_t0, box_nw, box_nt;
    float w[kWWCap];           // per depo: nt + 1 tick edges, then np + 1 impact edges
    float val[kWItemCap];
    typename Acc<DET>::T box[kWBoxCap];
    int tgt[kWItemCap];        // box or grid index of each cached item, -1 off the grid
    uint8_t slot[kWWCap];      // depo of each edge, then of each cached item
};

template <bool DET>
__device__ __forceinline__ void raster_warp(WarpSmem<DET> &S, const float *__restrict__ t0, const float *__restrict__ x,
                                            const float *__restrict__ y, const float *__restrict__ z,
                                            const float *__restrict__ q, int64_t n, const PlaneParams &pp,
                                            uint32_t event_lo, typename Acc<DET>::T *__restrict__ grid, int32_t *status,
                                            int64_t chunk, const uint32_t (&RK)[20], uint32_t *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t c0 = chunk * kWarpDepos;
    if (c0 >= n) return;
    const int cn = (int)((n - c0) < kWarpDepos ? (n - c0) : kWarpDepos);
    const uint32_t c3 = counter_c3(pp, event_lo);
    // per depo (lane < cn): window, its item / edge counts and clamped grid footprint
    int ni = 0, nwt = 0, fa0 = INT_MAX, fa1 = INT_MIN, fb0 = INT_MAX, fb1 = INT_MIN;
    if (lane < cn) {
        const int64_t i = c0 + lane;
        DepoDesc d;
        if (!depo_window(t0[i], x[i], y[i], z[i], q[i], pp, d)) set_status(status, ST_EINVAL);
        else d.q = drift_absorb(d.q, x[i], (uint32_t)i, event_lo, pp);
        S.d[lane] = d;
        int wl = 0, nw = 0;
        if (d.nt > 0) {
            wl = floor_div(d.lo_p, pp.n_imp);
            nw = floor_div(d.lo_p + d.np - 1, pp.n_imp) - wl + 1;
            ni = (int)d.nt * nw;
            nwt = (int)d.nt + (int)d.np + 2;
            const int a0 = max(wl, 0), a1 = min(wl + nw - 1, pp.n_wires - 1);
            const int b0 = max(d.lo_t, 0), b1 = min(d.lo_t + (int)d.nt - 1, pp.n_ticks - 1);
            if (a0 <= a1 && b0 <= b1) fa0 = a0, fa1 = a1, fb0 = b0, fb1 = b1;
        }
        S.wl[lane] = wl;
        S.nw[lane] = nw;
        mark_tiles(flags, pp, d, wl, nw);
        S.sum[lane] = 0.f;
    }
    // one pass for all cn depos when their items and edges fit (the common case): offsets by
    // warp prefix sums, footprint by warp reductions; otherwise lane 0 packs passes greedily
    int inc_i = ni, inc_w = nwt;
#pragma unroll
    for (int o = 1; o < kWarpDepos; o <<= 1) {
        const int vi = __shfl_up_sync(0xffffffffu, inc_i, o), vw = __shfl_up_sync(0xffffffffu, inc_w, o);
        if (lane >= o) inc_i += vi, inc_w += vw;
    }
    const int tot_i = __shfl_sync(0xffffffffu, inc_i, cn - 1), tot_w = __shfl_sync(0xffffffffu, inc_w, cn - 1);
    const bool one_pass = tot_i <= kWItemCap && tot_w <= kWWCap;
    if (one_pass) {
        const int w0 = __reduce_min_sync(0xffffffffu, fa0), w1 = __reduce_max_sync(0xffffffffu, fa1);
        const int t0b = __reduce_min_sync(0xffffffffu, fb0), t1b = __reduce_max_sync(0xffffffffu, fb1);
        if (lane < cn) {
            S.item_off[lane] = inc_i - ni;
            S.w_off[lane] = inc_w - nwt;
        }
        if (lane == 0) {
            S.item_off[cn] = tot_i;
            S.w_off[cn] = tot_w;
            S.pass_end = cn;
            const bool any = w0 <= w1;
            const int64_t area = any ? (int64_t)(w1 - w0 + 1) * (t1b - t0b + 1) : 0;
            S.use_box = any && area <= kWBoxCap;
            S.box_w0 = w0;
            S.box_t0 = t0b;
            S.box_nw = any ? w1 - w0 + 1 : 0;
            S.box_nt = any ? t1b - t0b + 1 : 0;
        }
    }
    __syncwarp();
    for (int s = 0; s < cn;) {
        if (lane == 0 && !one_pass) {
            int it = 0, ww = 0, e = s;
            int w0 = INT_MAX, w1 = INT_MIN, t0b = INT_MAX, t1b = INT_MIN;
            for (; e < cn; ++e) {
                const DepoDesc &d = S.d[e];
                const int ni = (int)d.nt * S.nw[e], nwt = d.nt > 0 ? (int)d.nt + (int)d.np + 2 : 0;
                if (e > s && (it + ni > kWItemCap || ww + nwt > kWWCap)) break;
                S.item_off[e] = it;
                S.w_off[e] = ww;
                it += ni;
                ww += nwt;
                if (d.nt > 0) {
                    const int a0 = max(S.wl[e], 0), a1 = min(S.wl[e] + S.nw[e] - 1, pp.n_wires - 1);
                    const int b0 = max(d.lo_t, 0), b1 = min(d.lo_t + (int)d.nt - 1, pp.n_ticks - 1);
                    if (a0 <= a1 && b0 <= b1) {
                        w0 = min(w0, a0); w1 = max(w1, a1);
                        t0b = min(t0b, b0); t1b = max(t1b, b1);
                    }
                }
            }
            S.item_off[e] = it;
            S.w_off[e] = ww;
            S.pass_end = e;
            const bool any = w0 <= w1;
            const int64_t area = any ? (int64_t)(w1 - w0 + 1) * (t1b - t0b + 1) : 0;
            S.use_box = any && area <= kWBoxCap;
            S.box_w0 = w0;
            S.box_t0 = t0b;
            S.box_nw = any ? w1 - w0 + 1 : 0;
            S.box_nt = any ? t1b - t0b + 1 : 0;
        }
        __syncwarp();
        const int e = S.pass_end;
        const int n_items = S.item_off[e] - S.item_off[s];
        const int i_base = S.item_off[s];
        const int n_w = S.w_off[e] - S.w_off[s];
        const int w_base = S.w_off[s];
        const bool use_box = S.use_box && WCT_IDX_OK(status, S.box_nw * S.box_nt - 1, kWBoxCap);
        const int bnt = S.box_nt, bw0 = S.box_w0, bt0 = S.box_t0;
        if (!WCT_IDX_OK(status, n_w, kWWCap + 1)) break;   // never: the pass planning caps n_w
        if (use_box)
            for (int k = lane; k < S.box_nw * bnt; k += 32) S.box[k] = 0;
        // depo of every edge (a table instead of a search)
        for (int j = s; j < e; ++j)
            for (int k = S.w_off[j] - w_base + lane; k < S.w_off[j + 1] - w_base; k += 32) S.slot[k] = (uint8_t)j;
        __syncwarp();
        // bin edges erf((i - mu) * inv), i = 0..n, per axis (a point charge: edges 0, 1)
        for (int k = lane; k < n_w; k += 32) {
            const int j = S.slot[k];
            const DepoDesc &d = S.d[j];
            const int r = w_base + k - S.w_off[j];
            float E;
            if (r <= d.nt) E = d.inv_t == 0.f ? (r == 0 ? 0.f : 1.f) : erff(((float)r - d.mu_t) * d.inv_t);
            else {
                const int rr = r - d.nt - 1;
                E = d.inv_p == 0.f ? (rr == 0 ? 0.f : 1.f) : erff(((float)rr - d.mu_p) * d.inv_p);
            }
            S.w[k] = E;
        }
        __syncwarp();
        if (lane < e - s && S.d[s + lane].nt > 0) {
            const int j = s + lane;
            const DepoDesc &d = S.d[j];
            const float *E = S.w + (S.w_off[j] - w_base);
            S.nrm_t[j] = 1.f / (E[d.nt] - E[0]);
            S.nrm_p[j] = 1.f / (E[d.nt + 1 + d.np] - E[d.nt + 1]);
        }
        __syncwarp();
        // weights (E[i + 1] - E[i]) * nrm in place of E[i]: tick weights at [0, nt), impact
        // weights at [nt + 1, nt + 1 + np) of each depo's block
        for (int base = 0; base < n_w; base += 32) {
            const int k = base + lane;
            float v = 0.f;
            bool wr = false;
            if (k < n_w) {
                const int j = S.slot[k];
                const int nt = S.d[j].nt;
                const int r = w_base + k - S.w_off[j];
                if (r != nt && r != nt + 1 + S.d[j].np) {
                    v = (S.w[k + 1] - S.w[k]) * (r < nt ? S.nrm_t[j] : S.nrm_p[j]);
                    wr = true;
                }
            }
            __syncwarp();
            if (wr) S.w[k] = v;
            __syncwarp();
        }
        // depo of every cached item
        for (int j = s; j < e; ++j) {
            const int i1 = min(S.item_off[j + 1] - i_base, kWItemCap);
            for (int k = S.item_off[j] - i_base + lane; k < i1; k += 32) S.slot[k] = (uint8_t)j;
        }
        __syncwarp();
        for (int base = 0; base < n_items; base += 32) {
            const int k = base + lane;
            int j = -1;
            float v = 0.f;
            if (k < n_items) {
                j = k < kWItemCap ? S.slot[k] : find_slot(S.item_off, s, e, i_base + k);
                const DepoDesc &d = S.d[j];
                const Item f = make_item(i_base + k - S.item_off[j], S.nw[j], S.wl[j], d, pp.n_imp);
                const float *wt = S.w + (S.w_off[j] - w_base);
                const float *wp = wt + d.nt + 1;
                v = pp.fluctuate ? fold_fluct(f, wt, wp, d.q, (uint32_t)(c0 + j), pp, c3, RK) : fold_plain(f, wt, wp, d.q);
                if (k < kWItemCap) {
                    S.val[k] = v;
                    const bool in = f.wire >= 0 && f.wire < pp.n_wires && f.tick >= 0 && f.tick < pp.n_ticks;
                    S.tgt[k] = !in ? -1 : (use_box ? (f.wire - bw0) * bnt + (f.tick - bt0) : f.wire * pp.n_ticks + f.tick);
                }
            }
            if (pp.fluctuate) segmented_add(j, v, S.sum);
        }
        __syncwarp();
        // each depo's fluctuated sum -> its rescale factor q / sum (-1: keep the unfluctuated patch)
        if (pp.fluctuate && lane < e - s) {
            const float sm = S.sum[s + lane];
            S.sum[s + lane] = sm > 0.f ? S.d[s + lane].q / sm : -1.f;
        }
        __syncwarp();
        // cached items: target, depo and value were stored by the pass above
        const int n_cached = min(n_items, kWItemCap);
        for (int k = lane; k < n_cached; k += 32) {
            const int t = S.tgt[k];
            if (t < 0) continue;
            const int j = S.slot[k];
            float v = S.val[k];
            if (pp.fluctuate) {
                const float sc = S.sum[j];
                if (sc > 0.f) {
                    v *= sc;
                } else {
                    const DepoDesc &d = S.d[j];
                    const Item f = make_item(i_base + k - S.item_off[j], S.nw[j], S.wl[j], d, pp.n_imp);
                    const float *wt = S.w + (S.w_off[j] - w_base);
                    v = fold_plain(f, wt, wt + d.nt + 1, d.q);
                }
            }
            if (use_box) {
                if (WCT_IDX_OK(status, t, S.box_nw * bnt)) Acc<DET>::add(&S.box[t], v);
            } else if (WCT_IDX_OK(status, t, (int64_t)pp.n_wires * pp.n_ticks)) {
                Acc<DET>::add(&grid[t], v);
            }
        }
        // items beyond the cache (a single very wide depo) are recomputed
        for (int k = kWItemCap + lane; k < n_items; k += 32) {
            const int j = find_slot(S.item_off, s, e, i_base + k);
            const DepoDesc &d = S.d[j];
            const Item f = make_item(i_base + k - S.item_off[j], S.nw[j], S.wl[j], d, pp.n_imp);
            if (f.wire < 0 || f.wire >= pp.n_wires || f.tick < 0 || f.tick >= pp.n_ticks) continue;
            const float *wt = S.w + (S.w_off[j] - w_base);
            float v = pp.fluctuate ? fold_fluct(f, wt, wt + d.nt + 1, d.q, (uint32_t)(c0 + j), pp, c3, RK)
                                   : fold_plain(f, wt, wt + d.nt + 1, d.q);
            if (pp.fluctuate) {
                const float sc = S.sum[j];
                if (sc > 0.f) v *= sc;
                else v = fold_plain(f, wt, wt + d.nt + 1, d.q);
            }
            if (use_box) {
                const int t = (f.wire - bw0) * bnt + (f.tick - bt0);
                if (WCT_IDX_OK(status, t, S.box_nw * bnt)) Acc<DET>::add(&S.box[t], v);
            } else {
                const int64_t t = (int64_t)f.wire * pp.n_ticks + f.tick;
                if (WCT_IDX_OK(status, t, (int64_t)pp.n_wires * pp.n_ticks)) Acc<DET>::add(&grid[t], v);
            }
        }
        __syncwarp();
        if (use_box) {
            const int area = S.box_nw * bnt;
            for (int k = lane; k < area; k += 32) {
                const auto v = S.box[k];
                if (v != 0) {
                    const int r = k / bnt;
                    const int64_t t = (int64_t)(bw0 + r) * pp.n_ticks + bt0 + (k - r * bnt);
                    if (WCT_IDX_OK(status, t, (int64_t)pp.n_wires * pp.n_ticks)) atomicAdd(&grid[t], v);
                }
            }
        }
        __syncwarp();
        s = e;
    }
}

template <bool DET>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_raster_warps(const float *__restrict__ t0, const float *__restrict__ x, const float *__restrict__ y,
               const float *__restrict__ z, const float *__restrict__ q, int64_t n, PlaneParams pp,
               uint32_t event_lo, typename Acc<DET>::T *__restrict__ grid, int32_t *status, uint32_t *flags) {
    __shared__ WarpSmem<DET> S[kWarpsPerCta];
    const int warp = threadIdx.x >> 5;
    raster_warp<DET>(S[warp], t0, x, y, z, q, n, pp, event_lo, grid, status, (int64_t)blockIdx.x * kWarpsPerCta + warp,
                     pp.rk, flags);
}

// Batched: warp-chunk c of the whole launch belongs to the (event, plane) pair whose chunk
// range (in warp-chunks) holds c.
template <bool DET>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_raster_batch_warps(const BatchTable tab, int32_t *status) {
    __shared__ WarpSmem<DET> S[kWarpsPerCta];
    const int warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    int lo = 0, hi = tab.n_items;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tab.item[mid].chunk_begin <= c) lo = mid;
        else hi = mid;
    }
    const BatchItem &it = tab.item[lo];
    // every plane shares the seed, hence the round keys: take them from plane 0 (static index)
    typename Acc<DET>::T *grid;
    if constexpr (DET) grid = it.grid64;
    else grid = it.grid;
    raster_warp<DET>(S[warp], it.t0, it.x, it.y, it.z, it.q, it.n, tab.plane[it.plane], it.event_lo, grid, status,
                     c - it.chunk_begin, tab.plane[0].rk, it.flags);
}

// Batched, persistent: one launch for every (event, plane) pair of a batch.  Each warp keeps
// taking the next warp-chunk from a device counter until the batch's chunks are exhausted, so
// no warp waits for its CTA's siblings and the launch has no tail of idle CTA slots; the pairs
// are ordered by the host (largest events first), so the most expensive chunks go out first.
template <bool DET>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_raster_batch_persistent(const BatchTable tab, int64_t total_chunks, unsigned long long *__restrict__ counter,
                          int32_t *status) {
    __shared__ WarpSmem<DET> S[kWarpsPerCta];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned long long)total_chunks) break;
        int lo = 0, hi = tab.n_items;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tab.item[mid].chunk_begin <= (int64_t)c) lo = mid;
            else hi = mid;
        }
        const BatchItem &it = tab.item[lo];
        typename Acc<DET>::T *grid;
        if constexpr (DET) grid = it.grid64;
        else grid = it.grid;
        raster_warp<DET>(S[warp], it.t0, it.x, it.y, it.z, it.q, it.n, tab.plane[it.plane], it.event_lo, grid, status,
                         (int64_t)c - it.chunk_begin, tab.plane[0].rk, it.flags);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kChunkThreads)
k_raster_chunks(const float *__restrict__ t0, const float *__restrict__ x, const float *__restrict__ y,
                const float *__restrict__ z, const float *__restrict__ q, int64_t n, PlaneParams pp,
                uint32_t event_lo, float *__restrict__ grid, int32_t *status, uint32_t *flags) {
    extern __shared__ float4 smem_raw[];
    ChunkSmem &S = *reinterpret_cast<ChunkSmem *>(smem_raw);
    raster_chunk(S, t0, x, y, z, q, n, pp, event_lo, grid, status, blockIdx.x, pp.rk, flags);
}

// Many (event, plane) pairs in one launch: CTA b takes chunk b - chunk_begin[i] of the pair i
// whose chunk range holds b.
__global__ void __launch_bounds__(kChunkThreads)
k_raster_batch(const BatchTable tab, int32_t *status) {
    extern __shared__ float4 smem_raw[];
    ChunkSmem &S = *reinterpret_cast<ChunkSmem *>(smem_raw);
    const int64_t b = blockIdx.x;
    int lo = 0, hi = tab.n_items;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tab.item[mid].chunk_begin <= b) lo = mid;
        else hi = mid;
    }
    const BatchItem &it = tab.item[lo];
    raster_chunk(S, it.t0, it.x, it.y, it.z, it.q, it.n, tab.plane[it.plane], it.event_lo, it.grid, status,
                 b - it.chunk_begin, tab.plane[0].rk, it.flags);
}

// ------------------------------------------------------------------------------------------
// Unfused: full patches, one warp per depo (grid-stride).  Patch row-major [tick][impact].
// ------------------------------------------------------------------------------------------
constexpr int kPatchWarps = 8;

__device__ __forceinline__ float bin_normal(const PlaneParams &pp, uint32_t depo, int tick, int impact, uint32_t c3) {
    const int G = (pp.n_imp + 3) >> 2;
    const int wire = floor_div(impact, pp.n_imp);
    const int sub = impact - wire * pp.n_imp;
    const int g = sub >> 2, l = sub & 3;
    const uint4 x = philox4x32_10(make_uint4(depo, (uint32_t)tick, (uint32_t)(wire * G + g), c3), pp.key0, pp.key1);
    const float2 p = (l < 2) ? box_muller(x.x, x.y) : box_muller(x.z, x.w);
    return (l & 1) ? p.y : p.x;
}

__global__ void __launch_bounds__(kPatchWarps * 32)
k_rasterize_patches(int64_t n, const DepoDesc *__restrict__ desc, const int64_t *__restrict__ offsets,
                    int64_t slot, PlaneParams pp, uint32_t event_lo, float *__restrict__ patches) {
    __shared__ float wbuf[kPatchWarps][kWBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wt = wbuf[warp];
    float *wp = wt + kWT;
    const uint32_t c3 = counter_c3(pp, event_lo);
    const int64_t nwarps = (int64_t)gridDim.x * kPatchWarps;
    for (int64_t di = (int64_t)blockIdx.x * kPatchWarps + warp; di < n; di += nwarps) {
        const DepoDesc d = desc[di];
        const int nt = d.nt, np = d.np;
        if (nt == 0) continue;
        axis_weights(wt, nt, d.mu_t, d.inv_t, lane);
        axis_weights(wp, np, d.mu_p, d.inv_p, lane);
        float *out = patches + (offsets ? offsets[di] : di * slot);
        const int bins = nt * np;
        const float q = d.q;
        if (!pp.fluctuate) {
            for (int b = lane; b < bins; b += 32) {
                const int a = b / np, j = b - a * np;
                out[b] = q * wt[a] * wp[j];
            }
        } else {
            float part = 0.f;
            for (int b = lane; b < bins; b += 32) {
                const int a = b / np, j = b - a * np;
                const float w = wt[a] * wp[j];
                const float m = q * w;
                const float z = bin_normal(pp, (uint32_t)di, d.lo_t + a, d.lo_p + j, c3);
                const float v = fmaxf(fmaf(sfu_sqrt(fmaf(-m, w, m)), z, m), 0.f);
                out[b] = v;
                part += v;
            }
            const float total = warp_sum(part);
            for (int b = lane; b < bins; b += 32) {   // same lane -> same bins as above
                const int a = b / np, j = b - a * np;
                out[b] = total > 0.f ? out[b] * (q / total) : q * wt[a] * wp[j];
            }
        }
        __syncwarp();
    }
}

__global__ void k_write_patch_desc(int64_t n, const DepoDesc *__restrict__ desc, const int64_t *__restrict__ offsets,
                                   int64_t slot, int64_t *__restrict__ pd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DepoDesc d = desc[i];
    int64_t *e = pd + 5 * i;
    e[0] = offsets ? offsets[i] : i * slot;
    e[1] = d.lo_t;
    e[2] = d.lo_p;
    e[3] = d.nt;
    e[4] = d.np;
}

// Scatter caller-supplied patches: CTA per tile, items (tick, wire) fold the patch row.  The
// tile is accumulated in shared memory (fixed point in the deterministic mode) and written once.
template <int TW, int TT, bool DET>
__global__ void __launch_bounds__(kTileWarps * 32)
k_tile_scatter_patches(const int64_t *__restrict__ pd, const float *__restrict__ patches,
                       const int32_t *__restrict__ tile_off, const int32_t *__restrict__ tile_list, int64_t list_cap,
                       PlaneParams pp, float *__restrict__ grid, int32_t *status) {
    extern __shared__ float4 smem4[];
    using T = typename Acc<DET>::T;
    T *tile = reinterpret_cast<T *>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile_id = blockIdx.x;
    const int tw = tile_id / pp.n_tiles_t;
    const int tt = tile_id - tw * pp.n_tiles_t;
    const int wire0 = tw * TW, tick0 = tt * TT;
    const int wire_end = min(wire0 + TW, pp.n_wires), tick_end = min(tick0 + TT, pp.n_ticks);
    for (int i = threadIdx.x; i < TW * TT; i += blockDim.x) tile[i] = 0;
    __syncthreads();
    const int beg = tile_off[tile_id];
    const int end = (int)min((int64_t)tile_off[tile_id + 1], list_cap);
    for (int li = beg + warp; li < end; li += kTileWarps) {
        const int di = tile_list[li];
        const int64_t *e = pd + 5 * (int64_t)di;
        const int64_t off = e[0];
        DepoDesc d;
        d.lo_t = (int32_t)e[1];
        d.lo_p = (int32_t)e[2];
        d.nt = (int16_t)e[3];
        d.np = (int16_t)e[4];
        const int nt = d.nt, np = d.np;
        const int wl = floor_div(d.lo_p, pp.n_imp);
        const int nw = floor_div(d.lo_p + np - 1, pp.n_imp) - wl + 1;
        const int items = nt * nw;
        for (int it = lane; it < items; it += 32) {
            const Item f = make_item(it, nw, wl, d, pp.n_imp);
            if (f.wire >= wire0 && f.wire < wire_end && f.tick >= tick0 && f.tick < tick_end) {
                const float *row = patches + off + (int64_t)f.a * np + f.j_base;
                float s = 0.f;
                for (int sub = f.sub_lo; sub < f.sub_hi; ++sub) s += row[sub];
                const int t = (f.wire - wire0) * TT + (f.tick - tick0);
                if (WCT_IDX_OK(status, t, TW * TT)) Acc<DET>::add(&tile[t], s);
            }
        }
    }
    __syncthreads();
    if constexpr (DET) {
        for (int i = threadIdx.x; i < TW * TT; i += blockDim.x) {
            const int r = i / TT, c = i - r * TT;
            const int wire = wire0 + r, tick = tick0 + c;
            if (wire < wire_end && tick < tick_end)
                grid[(int64_t)wire * pp.n_ticks + tick] = __ll2float_rn((long long)tile[i]) * (1.f / kFixScale);
        }
        return;
    }
    const bool vec = ((pp.n_ticks & 3) == 0) && ((reinterpret_cast<uintptr_t>(grid) & 15) == 0);
    for (int i = threadIdx.x; i < TW * TT / 4; i += blockDim.x) {
        const int r = i / (TT / 4);
        const int c = (i - r * (TT / 4)) * 4;
        const int wire = wire0 + r, tick = tick0 + c;
        if (wire >= wire_end || tick >= tick_end) continue;
        float *dst = grid + (int64_t)wire * pp.n_ticks + tick;
        const float4 v = smem4[i];
        if (vec) {
            *reinterpret_cast<float4 *>(dst) = v;
        } else {
            dst[0] = v.x;
            if (tick + 1 < tick_end) dst[1] = v.y;
            if (tick + 2 < tick_end) dst[2] = v.z;
            if (tick + 3 < tick_end) dst[3] = v.w;
        }
    }
}

__global__ void k_philox(const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n,
                         uint32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = reinterpret_cast<const uint4 *>(ctr)[i];
    reinterpret_cast<uint4 *>(out)[i] = philox4x32_10(c, k0, k1);
}

constexpr int kTileW = 32, kTileT = 256;


}  // namespace

int tile_wires() { return kTileW; }
int tile_ticks() { return kTileT; }

// Raster schedule (PlaneParams::raster_schedule): 0 = warp-level chunks (default), 1 = CTA-level
// chunks.
int64_t raster_chunk_count(int64_t n, int schedule) {
    return schedule == 1 ? (n + kChunk - 1) / kChunk : (n + kWarpDepos - 1) / kWarpDepos;
}

cudaError_t launch_raster_batch(const BatchTable &tab, int64_t total_chunks, int32_t *status, cudaStream_t s,
                                bool det) {
    if (total_chunks <= 0) return cudaSuccess;
    if (det || tab.plane[0].raster_schedule != 1) {
        const int64_t blocks = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
        if (det) k_raster_batch_warps<true><<<(unsigned)blocks, kWarpsPerCta * 32, 0, s>>>(tab, status);
        else k_raster_batch_warps<false><<<(unsigned)blocks, kWarpsPerCta * 32, 0, s>>>(tab, status);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(ChunkSmem);
    cudaError_t e = cudaFuncSetAttribute(k_raster_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_raster_batch<<<(unsigned)total_chunks, kChunkThreads, smem, s>>>(tab, status);
    return cudaGetLastError();
}

namespace {
// CTAs of the persistent batch rasterizer resident on the whole current device, per device
// and accumulation mode, computed once under a lock.
constexpr int kMaxDevicesRaster = 64;
std::mutex g_raster_mu;
int g_raster_resident[kMaxDevicesRaster][2] = {};

int raster_resident(bool det) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesRaster ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 152;
    }
    std::lock_guard<std::mutex> lock(g_raster_mu);
    int &r = g_raster_resident[dev][det ? 1 : 0];
    if (r == 0) {
        int per_sm = 0;
        const cudaError_t e =
            det ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_batch_persistent<true>, kWarpsPerCta * 32, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_batch_persistent<false>, kWarpsPerCta * 32, 0);
        if (e != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        r = per_sm * sms;
    }
    return r;
}
}  // namespace

cudaError_t launch_raster_batch_persistent(const BatchTable &tab, int64_t total_chunks, unsigned long long *counter,
                                           int32_t *status, cudaStream_t s, bool det) {
    if (total_chunks <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t want = (total_chunks + kWarpsPerCta - 1) / kWarpsPerCta;
    const int64_t grid = std::min<int64_t>(want, raster_resident(det));
    if (det) k_raster_batch_persistent<true><<<(unsigned)grid, kWarpsPerCta * 32, 0, s>>>(tab, total_chunks, counter, status);
    else k_raster_batch_persistent<false><<<(unsigned)grid, kWarpsPerCta * 32, 0, s>>>(tab, total_chunks, counter, status);
    return cudaGetLastError();
}

cudaError_t launch_raster_chunks(const wct_depos_t &d, const PlaneParams &pp, uint32_t event_lo, float *grid,
                                 int32_t *status, cudaStream_t s, uint32_t *flags, unsigned long long *grid64) {
    if (d.n <= 0) return cudaSuccess;
    if (grid64 || pp.raster_schedule != 1) {
        const int64_t chunks = (d.n + kWarpDepos - 1) / kWarpDepos;
        const int64_t blocks = (chunks + kWarpsPerCta - 1) / kWarpsPerCta;
        if (grid64)
            k_raster_warps<true><<<(unsigned)blocks, kWarpsPerCta * 32, 0, s>>>(d.t0_us, d.x_mm, d.y_mm, d.z_mm, d.q_e,
                                                                                d.n, pp, event_lo, grid64, status, flags);
        else
            k_raster_warps<false><<<(unsigned)blocks, kWarpsPerCta * 32, 0, s>>>(d.t0_us, d.x_mm, d.y_mm, d.z_mm, d.q_e,
                                                                                 d.n, pp, event_lo, grid, status, flags);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(ChunkSmem);
    cudaError_t e = cudaFuncSetAttribute(k_raster_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (d.n + kChunk - 1) / kChunk;
    k_raster_chunks<<<(unsigned)blocks, kChunkThreads, smem, s>>>(d.t0_us, d.x_mm, d.y_mm, d.z_mm, d.q_e, d.n, pp,
                                                                  event_lo, grid, status, flags);
    return cudaGetLastError();
}

// Impact mode, fused: one warp per depo (grid-stride) evaluates its patch at impact resolution
// and adds every bin straight to the phase grid of its sub-bin (grid[phase][wire][tick], phase
// = the sub-bin's position inside its wire), with no patch buffer and no size query.  The work
// is flattened over (tick, wire, group of four sub-bins) units, one Philox call each, as the
// counter defines the groups.  With fluctuation the bins are drawn twice: once for the
// patch's fluctuated sum, once more to add them rescaled to the depo's charge.
template <bool DET>
__global__ void __launch_bounds__(kPatchWarps * 32)
k_raster_phases(int64_t n, const DepoDesc *__restrict__ desc, PlaneParams pp, uint32_t event_lo,
                typename Acc<DET>::T *__restrict__ grids, uint32_t *flags, int32_t *status) {
    __shared__ float wbuf[kPatchWarps][kWBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wt = wbuf[warp];
    float *wp = wt + kWT;
    const uint32_t c3 = counter_c3(pp, event_lo);
    const int n_imp = pp.n_imp, G = (n_imp + 3) >> 2;
    const int64_t nwarps = (int64_t)gridDim.x * kPatchWarps;
    for (int64_t di = (int64_t)blockIdx.x * kPatchWarps + warp; di < n; di += nwarps) {
        const DepoDesc d = desc[di];
        const int nt = d.nt, np = d.np;
        if (nt == 0) continue;
        axis_weights(wt, nt, d.mu_t, d.inv_t, lane);
        axis_weights(wp, np, d.mu_p, d.inv_p, lane);
        const int lo_p = d.lo_p, hi_p = d.lo_p + np;
        const int wl = floor_div(lo_p, n_imp);
        const int nw = floor_div(hi_p - 1, n_imp) - wl + 1;
        // groups per tick row: the first wire's (it may start inside a group), G for interior
        // wires, the last wire's (it may end inside one)
        const int sub_lo0 = lo_p - wl * n_imp, g_lo0 = sub_lo0 >> 2;
        const int cnt0 = ((min(n_imp, hi_p - wl * n_imp) - 1) >> 2) - g_lo0 + 1;
        const int cnt_l = nw > 1 ? ((hi_p - (wl + nw - 1) * n_imp - 1) >> 2) + 1 : 0;
        const int GD = cnt0 + (nw > 2 ? (nw - 2) * G : 0) + cnt_l;
        const int U = nt * GD;
        const float q = d.q;
        if (flags) {
            // the phase grids form one grid of n_imp * n_wires rows: flag the tiles under this
            // window in every phase's rows
            const int a0 = max(wl, 0), a1 = min(wl + nw - 1, pp.n_wires - 1);
            const int b0 = max(d.lo_t, 0), b1 = min(d.lo_t + nt - 1, pp.n_ticks - 1);
            const int n_tiles_w = (n_imp * pp.n_wires + pp.tile_w - 1) / pp.tile_w;
            if (a0 <= a1 && b0 <= b1)
                for (int ph = lane; ph < n_imp; ph += 32)
                    flag_tiles(flags, n_tiles_w * pp.n_tiles_t, pp.n_tiles_t, pp.tile_w, pp.tile_t, ph * pp.n_wires + a0,
                               ph * pp.n_wires + a1, b0, b1);
        }
        // unit u -> (window tick a, wire, group g) and its lanes [l0, l1) of the group
        auto unit = [&](int u, int &a, int &wire, int &g, int &l0, int &l1) {
            a = u / GD;
            const int r = u - a * GD;
            int w;
            if (r < cnt0) {
                w = 0;
                g = g_lo0 + r;
            } else {
                const int r2 = r - cnt0;
                w = 1 + r2 / G;
                g = r2 - (w - 1) * G;
            }
            wire = wl + w;
            const int first = wire * n_imp;
            const int sb = g << 2;
            l0 = max(max(first, lo_p) - first - sb, 0);
            l1 = min(min(first + n_imp, hi_p) - first - sb, 4);
        };
        auto draw = [&](int a, int wire, int g, float (&z)[4]) {
            const uint4 x = philox4x32_10_rk(make_uint4((uint32_t)di, (uint32_t)(d.lo_t + a), (uint32_t)(wire * G + g), c3),
                                             pp.rk);
            const float2 p0 = box_muller(x.x, x.y), p1 = box_muller(x.z, x.w);
            z[0] = p0.x, z[1] = p0.y, z[2] = p1.x, z[3] = p1.y;
        };
        float scale = 1.f;
        if (pp.fluctuate) {
            float part = 0.f;
            for (int u = lane; u < U; u += 32) {
                int a, wire, g, l0, l1;
                unit(u, a, wire, g, l0, l1);
                float z[4];
                draw(a, wire, g, z);
                const int jb = wire * n_imp + (g << 2) - lo_p;
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (l >= l0 && l < l1) {
                        const float w = wt[a] * wp[jb + l], m = q * w;
                        part += fmaxf(fmaf(sfu_sqrt(fmaf(-m, w, m)), z[l], m), 0.f);
                    }
            }
            const float sum = warp_sum(part);
            scale = sum > 0.f ? q / sum : -1.f;                 // -1: keep the unfluctuated patch
        }
        for (int u = lane; u < U; u += 32) {
            int a, wire, g, l0, l1;
            unit(u, a, wire, g, l0, l1);
            const int tick = d.lo_t + a;
            if (tick < 0 || tick >= pp.n_ticks || wire < 0 || wire >= pp.n_wires) continue;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (scale > 0.f && pp.fluctuate) draw(a, wire, g, z);
            const int jb = wire * n_imp + (g << 2) - lo_p;
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l >= l0 && l < l1) {
                    const float w = wt[a] * wp[jb + l], m = q * w;
                    const float v = (pp.fluctuate && scale > 0.f) ? fmaxf(fmaf(sfu_sqrt(fmaf(-m, w, m)), z[l], m), 0.f) * scale
                                                                 : m;
                    const int phase = (g << 2) + l;
                    const int64_t t = ((int64_t)phase * pp.n_wires + wire) * pp.n_ticks + tick;
                    if (WCT_IDX_OK(status, t, (int64_t)n_imp * pp.n_wires * pp.n_ticks)) Acc<DET>::add(&grids[t], v);
                }
        }
        __syncwarp();
    }
}

cudaError_t launch_raster_phases(int64_t n, const DepoDesc *desc, const PlaneParams &pp, uint32_t event_lo,
                                 float *grids, uint32_t *flags, cudaStream_t s, unsigned long long *grids64,
                                 int32_t *status) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + kPatchWarps - 1) / kPatchWarps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (grids64)
        k_raster_phases<true><<<(unsigned)blocks, kPatchWarps * 32, 0, s>>>(n, desc, pp, event_lo, grids64, flags, status);
    else
        k_raster_phases<false><<<(unsigned)blocks, kPatchWarps * 32, 0, s>>>(n, desc, pp, event_lo, grids, flags, status);
    return cudaGetLastError();
}

// Deterministic mode: the fixed-point tiles listed in `flags` (layout of flag_tiles; the list
// is only read) are added to the float grid, each value rounded once to float and scaled by
// 1 / kFixScale (exact), and zeroed again.  One CTA per listed tile, grid-stride; a thread per
// four adjacent bins (16-byte loads, several in flight) when the row length, the tile width and
// both grids allow it, else a thread per tick column.
__global__ void __launch_bounds__(256)
k_fix_tiles(const uint32_t *__restrict__ flags, int n_tiles, int n_tiles_t, int tile_w, int tile_t, int n_rows,
            int n_cols, unsigned long long *__restrict__ g64, float *__restrict__ grid, int32_t *status) {
    const uint32_t count = flags[n_tiles];
    // four bins per thread and several rows in flight where the rows allow 16-byte accesses
    const bool vec = (n_cols & 3) == 0 && (tile_t & 3) == 0 && (reinterpret_cast<uintptr_t>(grid) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(g64) & 15) == 0;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const int t = (int)flags[n_tiles + 2 + i];
        if (!WCT_IDX_OK(status, t, n_tiles)) continue;
        const int tw = t / n_tiles_t, tt = t - tw * n_tiles_t;
        const int r0 = tw * tile_w, c0 = tt * tile_t;
        const int r1 = min(r0 + tile_w, n_rows), c1 = min(c0 + tile_t, n_cols);
        if (vec) {
            const int q_per_row = (c1 - c0) >> 2;              // 4-bin quads per row of the tile
            const int n_q = (r1 - r0) * q_per_row;
#pragma unroll 4
            for (int k = threadIdx.x; k < n_q; k += blockDim.x) {
                const int r = r0 + k / q_per_row, c = c0 + 4 * (k - (k / q_per_row) * q_per_row);
                const size_t idx = (size_t)r * n_cols + c;
                ulonglong2 *g2 = reinterpret_cast<ulonglong2 *>(g64 + idx);
                const ulonglong2 a = g2[0], b = g2[1];
                if ((a.x | a.y | b.x | b.y) != 0ull) {
                    float4 *gf = reinterpret_cast<float4 *>(grid + idx);
                    float4 v = *gf;
                    const float sc = 1.f / kFixScale;
                    v.x += __ll2float_rn((long long)a.x) * sc;
                    v.y += __ll2float_rn((long long)a.y) * sc;
                    v.z += __ll2float_rn((long long)b.x) * sc;
                    v.w += __ll2float_rn((long long)b.y) * sc;
                    *gf = v;
                    g2[0] = make_ulonglong2(0ull, 0ull);
                    g2[1] = make_ulonglong2(0ull, 0ull);
                }
            }
            continue;
        }
        for (int r = r0; r < r1; ++r)
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                const size_t idx = (size_t)r * n_cols + c;
                const unsigned long long v = g64[idx];
                if (v != 0ull) {
                    grid[idx] += __ll2float_rn((long long)v) * (1.f / kFixScale);
                    g64[idx] = 0ull;
                }
            }
    }
}

cudaError_t launch_fix_tiles(const uint32_t *flags, int n_rows, int n_cols, int tile_w, int tile_t,
                             unsigned long long *g64, float *grid, cudaStream_t s, int32_t *status) {
    const int n_tiles_t = (n_cols + tile_t - 1) / tile_t;
    const int n_tiles = ((n_rows + tile_w - 1) / tile_w) * n_tiles_t;
    const int blocks = n_tiles < 2 * 152 ? n_tiles : 2 * 152;
    if (blocks <= 0) return cudaSuccess;
    k_fix_tiles<<<blocks, 256, 0, s>>>(flags, n_tiles, n_tiles_t, tile_w, tile_t, n_rows, n_cols, g64, grid, status);
    return cudaGetLastError();
}


// Size of a plane's flag block: the flags, two counters and the tile list.
size_t tile_flag_words(const PlaneParams &pp) { return 2 * (size_t)pp.n_tiles_w * pp.n_tiles_t + 2; }

ClearJob clear_job(float *grid, uint32_t *flags, const PlaneParams &pp) {
    ClearJob j;
    j.grid = grid;
    j.flags = flags;
    j.n_wires = pp.n_wires;
    j.n_ticks = pp.n_ticks;
    j.tile_w = pp.tile_w;
    j.tile_t = pp.tile_t;
    j.n_tiles_t = pp.n_tiles_t;
    j.n_tiles = pp.n_tiles_w * pp.n_tiles_t;
    return j;
}


cudaError_t launch_rasterize_patches(int64_t n, const DepoDesc *desc, const int64_t *offsets, const PlaneParams &pp,
                                     uint32_t event_lo, float *patches, int64_t *patch_desc, cudaStream_t s,
                                     int64_t slot) {
    if (n <= 0) return cudaSuccess;
    if (patch_desc) {
        k_write_patch_desc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, desc, offsets, slot, patch_desc);
    }
    if (patches) {
        int64_t blocks = (n + kPatchWarps - 1) / kPatchWarps;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_rasterize_patches<<<(unsigned)blocks, kPatchWarps * 32, 0, s>>>(n, desc, offsets, slot, pp, event_lo,
                                                                          patches);
    }
    return cudaGetLastError();
}

// Scan-free slots: a depo whose window holds more than `slot` bins is reported and emptied
// (nt = np = 0), so neither the patch kernel nor a scatter touches it.
__global__ void k_fit_slots(int64_t n, DepoDesc *__restrict__ desc, int64_t slot, int32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DepoDesc d = desc[i];
    if ((int64_t)d.nt * d.np > slot) {
        set_status(status, ST_EINVAL);
        d.nt = d.np = 0;
        desc[i] = d;
    }
}

cudaError_t launch_fit_slots(int64_t n, DepoDesc *desc, int64_t slot, int32_t *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fit_slots<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, desc, slot, status);
    return cudaGetLastError();
}

cudaError_t launch_tile_scatter_patches(const int64_t *patch_desc, const float *patches, const int32_t *tile_off,
                                        const int32_t *tile_list, int64_t list_cap, const PlaneParams &pp, float *grid,
                                        cudaStream_t s, bool det, int32_t *status) {
    const int n_tiles = pp.n_tiles_w * pp.n_tiles_t;
    if (n_tiles <= 0) return cudaSuccess;
    if (det) {
        const size_t smem = sizeof(unsigned long long) * (size_t)kTileW * kTileT;   // 64 KB
        auto kern = k_tile_scatter_patches<kTileW, kTileT, true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<n_tiles, kTileWarps * 32, smem, s>>>(patch_desc, patches, tile_off, tile_list, list_cap, pp, grid, status);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(float) * (size_t)kTileW * kTileT;
    k_tile_scatter_patches<kTileW, kTileT, false><<<n_tiles, kTileWarps * 32, smem, s>>>(
        patch_desc, patches, tile_off, tile_list, list_cap, pp, grid, status);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, k0, k1, n, out);
    return cudaGetLastError();
}

}  // namespace wct
