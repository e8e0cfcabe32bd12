// Host runtime and C ABI: handle, FFT plans, response spectra, scratch under an HBM budget,
// and the stream-ordered sequence of kernels for each entry point of include/wct_sim.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <atomic>
#include <vector>

#include "wct_internal.cuh"

namespace wct {
int tile_wires();
int tile_ticks();
}  // namespace wct

using namespace wct;

namespace {

constexpr int kMaxPlanes = 8;
constexpr int kStages = 5;        // prep + binning, raster-scatter, row r2c, wire stage, row c2r
constexpr int kMaxSlots = 4096;
constexpr int kMaxM = 14336;   // largest complex FFT length: two M-point buffers in one CTA's shared memory

struct PlaneState {
    wct_plane_t g{};
    PlaneParams pp{};
    FFTPlan fft{};
    float2 *resp_spec = nullptr;   // [WCT_MAX_RESPONSE_WIRES][Fs], scaled by 1/M
    int n_tiles = 0;
    int max_tiles_per_depo = 0;
    // impact mode (per-impact-position responses): one response spectrum per phase, stride
    // fft_imp.Fs = fft_imp.Fu (the union of the phases' supports), and n_phases phase grids
    int n_phases = 0;              // 0: folded mode
    FFTPlan fft_imp{};
    float2 *resp_imp = nullptr;    // [n_phases][WCT_MAX_RESPONSE_WIRES][fft_imp.Fs], scaled by 1/M
    size_t resp_imp_bytes = 0;
    float *phase_grids = nullptr;  // [n_phases][n_wires][n_ticks], all zero between events
    size_t phase_grid_bytes = 0;
    uint32_t *phase_flags = nullptr;   // touched-tile flags + list of the phase grids (one grid)
    size_t phase_flag_bytes = 0;
    uint8_t *phase_act = nullptr;      // row activity of the phase grids [n_phases][n_wires] + [n_wires]
    unsigned long long *phase_grids64 = nullptr;   // deterministic mode: fixed-point phase grids
    size_t phase_grid64_bytes = 0;
    int phase_tiles = 0;
    // coloured noise of the digitiser: amplitude per spectrum bin, spectrum and waveform scratch
    float *noise_amp = nullptr;
    float2 *noise_spec = nullptr;
    float *noise_wave = nullptr;
    size_t noise_bytes[3] = {0, 0, 0};
};

}  // namespace

struct wct_sim {
    int device = 0;
    int n_planes = 0;
    PlaneState planes[kMaxPlanes];
    wct_diffusion_t diff{};
    wct_opts_t opts{};
    // scratch
    float2 *spec = nullptr, *spec2 = nullptr;
    size_t spec_elems = 0;          // capacity of spec / spec2 (complex elements)
    float2 *spec_imp = nullptr;     // impact mode: the spectra of every phase [phase][wire][Fs]
    size_t spec_imp_elems = 0;

    // Accumulation grids: set 0 serves run_event, sets 1.. run_batch (one per event of a raster
    // launch, grown on demand).  A set holds every plane's grid and tile flags and is kept all
    // zero between uses: the rasterizer flags the tiles it touches, and once the forward
    // transform has read a grid those tiles are cleared again.
    std::vector<float *> grids;
    size_t grid_off[kMaxPlanes + 1] = {};
    std::vector<uint32_t *> tile_flags;
    size_t flag_off[kMaxPlanes + 1] = {};
    // Deterministic mode: the rasterizers accumulate fixed-point integers into grids64 (same
    // offsets as grids, all zero between uses) and launch_fix_tiles moves the touched tiles into
    // the float grid; det_flags lists the touched tiles when the target is a caller's grid.
    bool det = false;
    std::vector<unsigned long long *> grids64;
    uint32_t *det_flags = nullptr;
    // run_batch: work counter of the persistent raster launch, the second convolution stream's
    // spectrum scratch, and the events ordering the batch's streams
    unsigned long long *work_counter = nullptr;
    int batch_events_per_launch = 0;   // schedule: events per persistent raster launch (0 = all)
    int conv_streams = 2;              // schedule: convolution streams (1, 2 or 3)
    float2 *bspec[3][2] = {};          // convolution streams 1, 2: forward / wire-stage spectra
    size_t bspec_elems[3] = {};
    // per convolution scratch j (0: spec / spec2, j > 0: bspec[j]): the row activity of the grid
    // being convolved, act[j][0] its rows, act[j][1] the output rows (wct::launch_row_activity)
    uint8_t *act[3][2] = {};
    int max_wires = 0;
    std::vector<cudaEvent_t> evpool;
    DepoDesc *desc = nullptr;
    int64_t *patch_size = nullptr, *patch_off = nullptr, *scan64 = nullptr;
    int64_t depo_cap = 0;
    int32_t *tile_count = nullptr, *tile_off = nullptr, *tile_cursor = nullptr, *scan32 = nullptr;
    int32_t *tile_list = nullptr;
    int64_t list_cap = 0;
    int32_t *status = nullptr;
    size_t bytes = 0;
    std::vector<std::pair<void *, size_t>> allocs;   // live device allocations and their sizes
    std::string err;
    // stage timing: one slot of kStages + 1 events per (run_event call, plane)
    bool timing = false;
    std::vector<std::array<cudaEvent_t, kStages + 1>> slots;
    int slots_used = 0;
    int events_timed = 0;
    // run_batch timing, per raster launch: raster begin / end on the raster stream, then the
    // convolutions' begin / end on each convolution stream
    std::vector<std::array<cudaEvent_t, 6>> bslots;
    int bslots_used = 0;
    int batches_timed = 0;
    int64_t launches = 0;   // kernels launched by this handle
    // run_batch: CUDA graphs of whole batches, keyed by the batch's pointers and sizes
    cudaStream_t cap_stream = nullptr;
    cudaStream_t rs_stream = nullptr, cv_stream[3] = {};   // run_batch raster / convolution streams
    struct Graph {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec;
        int64_t kernels;   // kernels recorded in the graph
    };
    std::vector<Graph> graphs;
    std::vector<std::vector<uint64_t>> seen;   // recent batch keys not (yet) recorded
    int64_t graph_launches = 0;
    // run_event: the planes' convolutions forked onto two streams of the caller's priority
    // (one pair per priority seen), ordered by ev_plane (a plane's grid is complete) and
    // ev_join (a fork stream's work is done); ev_overlap_off after scratch could not be had
    struct EventStreams {
        int priority;
        cudaStream_t st[2];
    };
    std::vector<EventStreams> ev_streams;
    cudaEvent_t ev_plane[kMaxPlanes] = {}, ev_join[2] = {};
    bool ev_overlap_off = false;
    // run_host: upload / compute / download streams, double-buffered device staging
    cudaStream_t up_stream = nullptr, comp_stream = nullptr, down_stream = nullptr;
    cudaEvent_t ev_up[2] = {}, ev_comp[2] = {}, ev_down[2] = {};
    float *h_depo[2] = {};                  // 5 arrays of h_cap floats each
    int64_t h_cap = 0;
    float *h_wave[2][kMaxPlanes] = {};
};

namespace {

wct_status_t fail(wct_sim *s, wct_status_t code, const std::string &msg) {
    if (s) s->err = msg;
    return code;
}

wct_status_t cuda_fail(wct_sim *s, cudaError_t e, const char *where) {
    return fail(s, WCT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Armed by wct_debug_fail_alloc: the allocation that finds the count at 0 fails (-1: disarmed).
std::atomic<long long> g_fail_alloc{-1};

bool injected_alloc_failure() {
    long long k = g_fail_alloc.load(std::memory_order_relaxed);
    while (k >= 0)
        if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 0;
    return false;
}

wct_status_t dev_alloc(wct_sim *s, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_alloc_failure()) return fail(s, WCT_ENOMEM, "injected allocation failure");
    if (s->opts.hbm_budget_bytes && s->bytes + bytes > s->opts.hbm_budget_bytes)
        return fail(s, WCT_ENOMEM, "scratch would exceed the HBM budget");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(s, WCT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    s->bytes += bytes;
    s->allocs.emplace_back(*p, bytes);
    return WCT_OK;
}

// Free one allocation (null: nothing); the size accounted is the one recorded at allocation.
void dev_free(wct_sim *s, void *p, size_t /*bytes*/ = 0) {
    if (!p) return;
    cudaFree(p);
    for (auto &a : s->allocs)
        if (a.first == p) {
            s->bytes -= a.second;
            a = {nullptr, 0};
        }
}

// Allocate every (pointer, bytes) pair or none: after a failure the ones already taken are
// freed again and every pointer of the set is null.
wct_status_t dev_alloc_all(wct_sim *s, std::initializer_list<std::pair<void **, size_t>> set) {
    wct_status_t st = WCT_OK;
    for (const auto &a : set)
        if ((st = dev_alloc(s, a.first, a.second)) != WCT_OK) break;
    if (st != WCT_OK)
        for (const auto &a : set) {
            dev_free(s, *a.first);
            *a.first = nullptr;
        }
    return st;
}

bool smooth7(int64_t m) {
    for (int p : {2, 3, 5, 7})
        while (m % p == 0) m /= p;
    return m == 1;
}

// Highest bin f < F whose exact DFT (length P, FP64) of some response row exceeds `thr` in
// magnitude; scans down from the top and stops at the first such bin (0 if none).
int response_support_last(const wct_response_t &r, int P, int F, double thr) {
    std::vector<double> c(P), sn(P);
    for (int j = 0; j < P; ++j) {
        const double a = 2.0 * M_PI * (double)j / (double)P;
        c[j] = std::cos(a);
        sn[j] = std::sin(a);
    }
    const double thr2 = thr * thr;
    for (int f = F - 1; f > 0; --f)
        for (int row = 0; row < r.n_wires_resp; ++row) {
            const float *x = r.host_data + (size_t)row * r.n_ticks_resp;
            double re = 0.0, im = 0.0;
            int64_t j = 0;
            for (int n = 0; n < r.n_ticks_resp; ++n) {
                re += (double)x[n] * c[j];
                im -= (double)x[n] * sn[j];
                j += f;
                if (j >= P) j -= P;
            }
            if (re * re + im * im > thr2) return f;
        }
    return 0;
}

constexpr int kNumRadices = 6;
// Row-transform schedule of a handle created with schedule_id -1 (FFTPlan::row_schedule)
constexpr int kDefaultRowSchedule = 3;

// Shared-memory wavefronts of one Stockham stage (radix R after stages of product NS) for a
// length-M transform: each warp handles 32 consecutive butterflies j, reads its R inputs
// x[j + r M/R] (contiguous), one twiddle tw[(j mod NS) M/(NS R)] and writes its R outputs to
// (j - j mod NS) R + j mod NS + r NS.  A 64-bit access costs, per bank (32 banks of 4 bytes),
// one wavefront per distinct word the warp touches there.
int64_t stage_wavefronts(int M, int R, int NS) {
    const int NB = M / R, stride = M / (NS * R);
    int64_t total = 0;
    int64_t addr[32];
    auto cost = [&](int n) {
        int words[32][64];
        int nw[32] = {0};
        int worst = 0;
        for (int l = 0; l < n; ++l)
            for (int h = 0; h < 2; ++h) {
                const int64_t w = 2 * addr[l] + h;
                const int b = (int)(w % 32);
                bool seen = false;
                for (int i = 0; i < nw[b]; ++i) seen |= words[b][i] == (int)w;
                if (!seen) words[b][nw[b]++] = (int)w;
                worst = std::max(worst, nw[b]);
            }
        return (int64_t)worst;
    };
    for (int w0 = 0; w0 < NB; w0 += 32) {
        const int n = std::min(32, NB - w0);
        for (int rr = 0; rr < R; ++rr) {
            for (int l = 0; l < n; ++l) addr[l] = w0 + l + (int64_t)rr * NB;
            total += cost(n);
        }
        if (NS > 1) {
            for (int l = 0; l < n; ++l) addr[l] = (int64_t)((w0 + l) % NS) * stride;
            total += cost(n);
        }
        for (int rr = 0; rr < R; ++rr) {
            for (int l = 0; l < n; ++l) {
                const int j = w0 + l, k = j % NS;
                addr[l] = (int64_t)(j - k) * R + k + (int64_t)rr * NS;
            }
            total += cost(n);
        }
    }
    return total;
}

// Stage order with the fewest shared-memory wavefronts under stage_wavefronts: dynamic
// programming over the sub-multisets of radices already applied (the next stage's cost
// depends only on its radix and the product of those before it).
void order_stages(int M, const int rads[kNumRadices], const int count[kNumRadices], int32_t *out) {
    int dims[kNumRadices], n_states = 1;
    for (int i = 0; i < kNumRadices; ++i) {
        dims[i] = count[i] + 1;
        n_states *= dims[i];
    }
    auto decode = [&](int s, int *c) {
        for (int i = 0; i < kNumRadices; ++i) {
            c[i] = s % dims[i];
            s /= dims[i];
        }
    };
    auto encode = [&](const int *c) {
        int s = 0;
        for (int i = kNumRadices - 1; i >= 0; --i) s = s * dims[i] + c[i];
        return s;
    };
    const int64_t inf = INT64_MAX / 4;
    std::vector<int64_t> best(n_states, inf);
    std::vector<int> from(n_states, -1), via(n_states, -1);
    best[0] = 0;
    for (int s = 0; s < n_states; ++s) {            // states in increasing code: predecessors first
        if (best[s] >= inf) continue;
        int c[kNumRadices];
        decode(s, c);
        int NS = 1;
        for (int i = 0; i < kNumRadices; ++i)
            for (int k = 0; k < c[i]; ++k) NS *= rads[i];
        for (int i = 0; i < kNumRadices; ++i) {
            if (c[i] == count[i]) continue;
            ++c[i];
            const int t = encode(c);
            --c[i];
            const int64_t v = best[s] + stage_wavefronts(M, rads[i], NS);
            if (v < best[t]) {
                best[t] = v;
                from[t] = s;
                via[t] = rads[i];
            }
        }
    }
    std::vector<int> seq;
    for (int s = n_states - 1; s > 0; s = from[s]) seq.push_back(via[s]);
    for (size_t k = 0; k < seq.size(); ++k) out[k] = seq[seq.size() - 1 - k];
}

// FFT length: the smallest even P >= n_ticks + n_resp_ticks - 1 with P / 2 7-smooth, so
// the circular convolution of length P equals the linear one on the kept ticks.
bool plan_fft(int n_ticks, int kt, FFTPlan &p) {
    const int64_t need = (int64_t)n_ticks + kt - 1;
    int64_t M = (need + 1) / 2;
    while (!smooth7(M)) ++M;
    if (M > kMaxM) return false;
    p.M = (int32_t)M;
    p.fft_len = (int32_t)(2 * M);
    p.F = (int32_t)(M + 1);
    p.Fs = (int32_t)((M + 2) & ~1LL);
    p.Fu = p.Fs;
    p.row_schedule = kDefaultRowSchedule;
    // radix multiset: largest radices first (fewest stages); their order is chosen below
    int64_t r = M;
    const int rads[kNumRadices] = {8, 7, 5, 4, 3, 2};
    int count[kNumRadices] = {0, 0, 0, 0, 0, 0};
    int ns = 0;
    for (int rad : {8, 4, 7, 5, 3, 2}) {
        while (r % rad == 0) {
            if (++ns > 12) return false;
            for (int i = 0; i < kNumRadices; ++i)
                if (rads[i] == rad) ++count[i];
            r /= rad;
        }
    }
    if (r != 1) return false;
    order_stages((int)M, rads, count, p.radix);
    p.n_stages = ns;
    p.radix_code = 0;
    for (int k = 0; k < ns; ++k) p.radix_code |= (uint64_t)p.radix[k] << (4 * k);
    return true;
}

wct_status_t upload_twiddles(wct_sim *s, FFTPlan &p) {
    std::vector<float2> tw(p.M), rtw(p.M + 1);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < p.M; ++k) {
        const double a = -2.0 * pi * (double)k / (double)p.M;
        tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int k = 0; k <= p.M; ++k) {
        const double a = -2.0 * pi * (double)k / (double)p.fft_len;
        rtw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    wct_status_t st = dev_alloc(s, (void **)&p.tw, sizeof(float2) * tw.size());
    if (st) return st;
    st = dev_alloc(s, (void **)&p.rtw, sizeof(float2) * rtw.size());
    if (st) return st;
    cudaError_t e = cudaMemcpy(p.tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.rtw, rtw.data(), sizeof(float2) * rtw.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(s, e, "twiddle upload");
    return WCT_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

wct_status_t check_depos(wct_sim *s, const wct_depos_t *d) {
    if (!d) return fail(s, WCT_EINVAL, "depos is NULL");
    if (d->n < 0) return fail(s, WCT_EINVAL, "negative depo count");
    if (d->n > (int64_t)1 << 30) return fail(s, WCT_EINVAL, "more than 2^30 depos in one call");
    if (d->n > 0 && (!d->t0_us || !d->x_mm || !d->y_mm || !d->z_mm || !d->q_e))
        return fail(s, WCT_EINVAL, "a depo array pointer is NULL");
    return WCT_OK;
}

wct_status_t ensure_depo_capacity(wct_sim *s, int64_t n) {
    if (n <= s->depo_cap) return WCT_OK;
    int64_t cap = n < 1024 ? 1024 : n;
    if (s->depo_cap) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(s, e, "sync before scratch growth");
        dev_free(s, s->desc, sizeof(DepoDesc) * s->depo_cap);
        dev_free(s, s->patch_size, sizeof(int64_t) * s->depo_cap);
        dev_free(s, s->patch_off, sizeof(int64_t) * (s->depo_cap + 1));
        dev_free(s, s->scan64, sizeof(int64_t) * scan_tmp_elems(s->depo_cap));
        dev_free(s, s->tile_list, sizeof(int32_t) * s->list_cap);
        s->desc = nullptr;
        s->patch_size = s->patch_off = s->scan64 = nullptr;
        s->tile_list = nullptr;
        s->depo_cap = 0;
        s->list_cap = 0;
    }
    int per = 1;
    for (int p = 0; p < s->n_planes; ++p) per = std::max(per, s->planes[p].max_tiles_per_depo);
    const wct_status_t st = dev_alloc_all(s, {{(void **)&s->desc, sizeof(DepoDesc) * cap},
                                              {(void **)&s->patch_size, sizeof(int64_t) * cap},
                                              {(void **)&s->patch_off, sizeof(int64_t) * (cap + 1)},
                                              {(void **)&s->scan64, sizeof(int64_t) * scan_tmp_elems(cap)},
                                              {(void **)&s->tile_list, sizeof(int32_t) * cap * per}});
    if (st) return st;
    s->depo_cap = cap;
    s->list_cap = cap * per;
    return WCT_OK;
}

PlaneParams plane_params(const wct_sim *s, int p) {
    PlaneParams pp = s->planes[p].pp;
    return pp;
}

wct_status_t plane_check(wct_sim *s, int plane) {
    if (!s) return WCT_EINVAL;
    if (plane < 0 || plane >= s->n_planes) return fail(s, WCT_EINVAL, "plane index out of range");
    return WCT_OK;
}

// Index of a fresh timing slot (events created on first use), or -1 when not timing.
int acquire_slot(wct_sim *s) {
    if (!s->timing) return -1;
    if (s->slots_used >= kMaxSlots) return -1;
    if (s->slots_used == (int)s->slots.size()) {
        std::array<cudaEvent_t, kStages + 1> ev{};
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
        s->slots.push_back(ev);
    }
    return s->slots_used++;
}

void mark(wct_sim *s, int slot, int k, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(s->slots[slot][k], st);
}

// A fresh run_batch timing slot (one per raster launch), or -1 when not timing.
int acquire_batch_slot(wct_sim *s) {
    if (!s->timing || s->bslots_used >= kMaxSlots) return -1;
    if (s->bslots_used == (int)s->bslots.size()) {
        std::array<cudaEvent_t, 6> ev{};
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
        s->bslots.push_back(ev);
    }
    return s->bslots_used++;
}

void bmark(wct_sim *s, int slot, int k, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(s->bslots[slot][k], st);
}

// Restore the all-zero library grids after a failed call (synchronous; best effort).
void clear_grids(wct_sim *s) {
    for (size_t b = 0; b < s->grids.size(); ++b) {
        if (s->grids[b]) cudaMemset(s->grids[b], 0, sizeof(float) * s->grid_off[s->n_planes]);
        if (b < s->grids64.size() && s->grids64[b])
            cudaMemset(s->grids64[b], 0, sizeof(unsigned long long) * s->grid_off[s->n_planes]);
        if (s->tile_flags[b]) cudaMemset(s->tile_flags[b], 0, sizeof(uint32_t) * s->flag_off[s->n_planes]);
    }
    for (int p = 0; p < s->n_planes; ++p) {
        const PlaneState &ps = s->planes[p];
        if (ps.phase_grids) cudaMemset(ps.phase_grids, 0, ps.phase_grid_bytes);
        if (ps.phase_grids64) cudaMemset(ps.phase_grids64, 0, ps.phase_grid64_bytes);
        if (ps.phase_flags) cudaMemset(ps.phase_flags, 0, ps.phase_flag_bytes);
    }
    if (s->det_flags) cudaMemset(s->det_flags, 0, sizeof(uint32_t) * s->flag_off[s->n_planes]);
    cudaDeviceSynchronize();
}

// One more accumulation grid set (every plane's grid, tile flags and, in the deterministic
// mode, fixed-point grid), all zero; all or nothing.  Synchronous.
wct_status_t add_grid_set(wct_sim *s) {
    const size_t cells = s->grid_off[s->n_planes], words = s->flag_off[s->n_planes];
    float *g = nullptr;
    uint32_t *f = nullptr;
    unsigned long long *g64 = nullptr;
    wct_status_t st = s->det ? dev_alloc_all(s, {{(void **)&g, sizeof(float) * cells},
                                                 {(void **)&f, sizeof(uint32_t) * words},
                                                 {(void **)&g64, sizeof(unsigned long long) * cells}})
                             : dev_alloc_all(s, {{(void **)&g, sizeof(float) * cells}, {(void **)&f, sizeof(uint32_t) * words}});
    if (st) return st;
    cudaError_t e = cudaMemset(g, 0, sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMemset(f, 0, sizeof(uint32_t) * words);
    if (e == cudaSuccess && g64) e = cudaMemset(g64, 0, sizeof(unsigned long long) * cells);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dev_free(s, g);
        dev_free(s, f);
        dev_free(s, g64);
        return cuda_fail(s, e, "grid init");
    }
    s->grids.push_back(g);
    s->tile_flags.push_back(f);
    s->grids64.push_back(g64);
    return WCT_OK;
}

// Fused rasterize + scatter of one plane into `grid` (zeroed first unless it is known to be
// zero, then accumulated).
// Deterministic mode: into the fixed-point grid of grid set `gset`, then the touched tiles into
// `grid` (listed in `flags`, or in det_flags, reset afterwards, when the grid is the caller's).
wct_status_t raster_scatter(wct_sim *s, int plane, const wct_depos_t *d, float *grid, cudaStream_t st, int slot,
                            bool clear = true, uint32_t *flags = nullptr, int gset = 0) {
    const PlaneState &ps = s->planes[plane];
    const PlaneParams pp = plane_params(s, plane);
    cudaError_t e = clear ? cudaMemsetAsync(grid, 0, sizeof(float) * (size_t)ps.g.n_wires * ps.g.n_ticks, st)
                          : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(s, e, "grid clear");
    mark(s, slot, 1, st);
    if (s->det) {
        unsigned long long *g64 = s->grids64[gset] + s->grid_off[plane];
        uint32_t *fl = flags ? flags : s->det_flags + s->flag_off[plane];
        e = launch_raster_chunks(*d, pp, (uint32_t)d->event_id, grid, s->status, st, fl, g64);
        if (e == cudaSuccess)
            e = launch_fix_tiles(fl, ps.g.n_wires, ps.g.n_ticks, pp.tile_w, pp.tile_t, g64, grid, st, s->status);
        if (e == cudaSuccess && !flags)
            e = cudaMemsetAsync(fl, 0, sizeof(uint32_t) * tile_flag_words(pp), st);
        s->launches += d->n > 0 ? 2 : 1;
    } else {
        e = launch_raster_chunks(*d, pp, (uint32_t)d->event_id, grid, s->status, st, flags);
        s->launches += d->n > 0 ? 1 : 0;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "raster-scatter");
    mark(s, slot, 2, st);
    return WCT_OK;
}

// The convolution of one plane.  clear_grid (== grid, a library grid) with its tile flags:
// the flagged tiles are zeroed once the forward transform has read the grid.
// The convolution of one plane, with spectrum scratch js (0: spec / spec2, 1 or 2: bspec[js]).
// clear_grid (== grid, a library grid) with its tile flags: rows of the grid that no depo
// touched are all zero, so the transforms skip them (row activity from the flags), and the
// flagged tiles are zeroed once the forward transform has read the grid.
wct_status_t convolve_plane(wct_sim *s, int plane, const float *grid, float *wf, cudaStream_t st, int slot,
                            float *clear_grid = nullptr, uint32_t *flags = nullptr, int js = 0) {
    const PlaneState &ps = s->planes[plane];
    const int nw = ps.g.n_wires, nt = ps.g.n_ticks;
    float2 *S = js == 0 ? s->spec : s->bspec[js][0], *T = js == 0 ? s->spec2 : s->bspec[js][1];
    const uint8_t *act_s = nullptr, *act_t = nullptr;
    cudaError_t e = cudaSuccess;
    if (clear_grid && s->act[js][0]) {
        e = launch_row_activity(flags, ps.pp.n_tiles_t, ps.pp.tile_w, nw, s->act[js][0], s->act[js][1], st);
        if (e != cudaSuccess) return cuda_fail(s, e, "row activity");
        act_s = s->act[js][0];
        act_t = s->act[js][1];
        s->launches += 1;
    }
    e = launch_row_r2c(ps.fft, grid, nt, nt, nw, S, st, s->status, act_s);
    if (e != cudaSuccess) return cuda_fail(s, e, "row r2c");
    mark(s, slot, 3, st);
    // the wire stage clears the grid tiles the rasterizer listed, as a side job
    const ClearJob job = clear_grid ? clear_job(clear_grid, flags, ps.pp) : ClearJob{};
    e = launch_wire_stage(ps.fft, S, ps.resp_spec, nw, T, st, s->status, clear_grid ? &job : nullptr, false, 1, act_s);
    if (e != cudaSuccess) return cuda_fail(s, e, "wire stage");
    mark(s, slot, 4, st);
    e = launch_row_c2r(ps.fft, T, nw, wf, nt, nt, st, s->status, act_t);
    if (e != cudaSuccess) return cuda_fail(s, e, "row c2r");
    s->launches += 3;
    mark(s, slot, 5, st);
    return WCT_OK;
}

// Time spectra of one response padded to 21 centred rows (scaled by 1/M), row stride full.Fs,
// in a new device buffer (KW x full.Fs); host copy in *host for the support computation.
wct_status_t response_spectrum(wct_sim *s, const FFTPlan &full, const wct_response_t &r, float2 **out,
                               std::vector<float2> &host) {
    const int KW = WCT_MAX_RESPONSE_WIRES;
    const int off = (KW - r.n_wires_resp) / 2;
    std::vector<float> pad((size_t)KW * r.n_ticks_resp, 0.f);
    for (int row = 0; row < r.n_wires_resp; ++row)
        std::memcpy(&pad[(size_t)(row + off) * r.n_ticks_resp], r.host_data + (size_t)row * r.n_ticks_resp,
                    sizeof(float) * r.n_ticks_resp);
    float *d_resp = nullptr;
    *out = nullptr;
    wct_status_t st = dev_alloc(s, (void **)&d_resp, sizeof(float) * pad.size());
    if (st == WCT_OK) st = dev_alloc(s, (void **)out, sizeof(float2) * (size_t)KW * full.Fs);
    if (st != WCT_OK) {
        dev_free(s, d_resp, sizeof(float) * pad.size());
        return st;
    }
    cudaError_t e = cudaMemcpy(d_resp, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_row_r2c(full, d_resp, r.n_ticks_resp, r.n_ticks_resp, KW, *out, 0);
    if (e == cudaSuccess) e = launch_scale_spectrum(*out, (int64_t)KW * full.Fs, 1.0f / (float)full.M, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(s, d_resp, sizeof(float) * pad.size());
    host.assign((size_t)KW * full.Fs, make_float2(0.f, 0.f));
    if (e == cudaSuccess) e = cudaMemcpy(host.data(), *out, sizeof(float2) * host.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "response spectrum");
    return WCT_OK;
}

double spectrum_max(const std::vector<float2> &h, const FFTPlan &full) {
    double m = 0.0;
    for (int k = 0; k < WCT_MAX_RESPONSE_WIRES; ++k)
        for (int f = 0; f < full.F; ++f) {
            const float2 v = h[(size_t)k * full.Fs + f];
            m = std::max(m, std::sqrt((double)v.x * v.x + (double)v.y * v.y));
        }
    return m;
}

// Free the impact-mode state of one plane.
void drop_impact(wct_sim *s, PlaneState &ps) {
    dev_free(s, ps.resp_imp, ps.resp_imp_bytes);
    dev_free(s, ps.phase_grids, ps.phase_grid_bytes);
    dev_free(s, ps.phase_flags, ps.phase_flag_bytes);
    dev_free(s, ps.phase_grids64, ps.phase_grid64_bytes);
    dev_free(s, ps.phase_act);
    ps.phase_act = nullptr;
    ps.phase_grids64 = nullptr;
    ps.phase_grid64_bytes = 0;
    ps.resp_imp = nullptr;
    ps.phase_grids = nullptr;
    ps.phase_flags = nullptr;
    ps.resp_imp_bytes = ps.phase_grid_bytes = ps.phase_flag_bytes = 0;
    ps.phase_tiles = 0;
    ps.n_phases = 0;
}

// The clearing side job of the phase grids (one grid of n_phases * n_wires rows).
ClearJob phase_clear_job(const PlaneState &ps) {
    ClearJob j;
    j.grid = ps.phase_grids;
    j.flags = ps.phase_flags;
    j.n_wires = ps.n_phases * ps.g.n_wires;
    j.n_ticks = ps.g.n_ticks;
    j.tile_w = ps.pp.tile_w;
    j.tile_t = ps.pp.tile_t;
    j.n_tiles_t = ps.pp.n_tiles_t;
    j.n_tiles = ps.phase_tiles;
    return j;
}

// The impact-mode hot path of one plane: windows, then every patch bin added to the phase
// grid of its sub-bin (fused, no patch buffer), every phase grid's rows transformed in one
// launch, one wire stage summing all phases' stencils, one inverse transform.
wct_status_t run_plane_impact(wct_sim *s, int p, const wct_depos_t *d, float *wf, cudaStream_t cs, int slot) {
    PlaneState &ps = s->planes[p];
    const int nw = ps.g.n_wires, nt = ps.g.n_ticks;
    const int64_t n = d->n;
    wct_status_t st = ensure_depo_capacity(s, n);
    if (st) return st;
    // the phase grids are all zero: the wire stage clears the tiles this event touches
    mark(s, slot, 0, cs);
    mark(s, slot, 1, cs);
    const PlaneParams pp = plane_params(s, p);
    cudaError_t e = launch_prep(*d, pp, s->desc, nullptr, nullptr, s->status, cs);
    if (e == cudaSuccess)
        e = launch_raster_phases(n, s->desc, pp, (uint32_t)d->event_id, ps.phase_grids, ps.phase_flags, cs,
                                 ps.phase_grids64, s->status);
    if (e == cudaSuccess && ps.phase_grids64)
        e = launch_fix_tiles(ps.phase_flags, ps.n_phases * nw, nt, pp.tile_w, pp.tile_t, ps.phase_grids64,
                             ps.phase_grids, cs, s->status);
    if (e != cudaSuccess) return cuda_fail(s, e, "phase raster");
    s->launches += (n > 0 ? 2 : 0) + (ps.phase_grids64 ? 1 : 0);
    mark(s, slot, 2, cs);
    // every phase grid's rows in one forward launch (rows no depo touched skipped), one wire
    // stage over all phases, one inverse transform
    const uint8_t *act_s = ps.phase_act, *act_t = ps.phase_act ? ps.phase_act + (size_t)ps.n_phases * nw : nullptr;
    if (act_s) {
        e = launch_row_activity(ps.phase_flags, ps.pp.n_tiles_t, ps.pp.tile_w, nw, ps.phase_act,
                                ps.phase_act + (size_t)ps.n_phases * nw, cs, ps.n_phases);
        if (e != cudaSuccess) return cuda_fail(s, e, "phase row activity");
        s->launches += 1;
    }
    e = launch_row_r2c(ps.fft_imp, ps.phase_grids, nt, nt, ps.n_phases * nw, s->spec_imp, cs, s->status, act_s);
    if (e != cudaSuccess) return cuda_fail(s, e, "phase transforms");
    mark(s, slot, 3, cs);
    const ClearJob job = phase_clear_job(ps);
    e = launch_wire_stage(ps.fft_imp, s->spec_imp, ps.resp_imp, nw, s->spec2, cs, s->status, &job, false,
                          ps.n_phases, act_s);
    if (e != cudaSuccess) return cuda_fail(s, e, "phase stencils");
    s->launches += 2;
    mark(s, slot, 4, cs);
    e = launch_row_c2r(ps.fft_imp, s->spec2, nw, wf, nt, nt, cs, s->status, act_t);
    if (e != cudaSuccess) return cuda_fail(s, e, "row c2r");
    s->launches += 1;
    mark(s, slot, 5, cs);
    return WCT_OK;
}

wct_status_t ensure_conv_spectra(wct_sim *s, int n);

// The two fork streams of run_event for the caller's stream priority (created on first use).
cudaError_t event_streams(wct_sim *s, cudaStream_t caller, cudaStream_t (&fs)[2]) {
    int prio = 0;
    cudaError_t e = cudaStreamGetPriority(caller, &prio);
    if (e != cudaSuccess) return e;
    for (const auto &es : s->ev_streams)
        if (es.priority == prio) {
            fs[0] = es.st[0];
            fs[1] = es.st[1];
            return cudaSuccess;
        }
    wct_sim::EventStreams es{prio, {nullptr, nullptr}};
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
        e = cudaStreamCreateWithPriority(&es.st[j], cudaStreamNonBlocking, prio);
    for (int p = 0; p < s->n_planes && e == cudaSuccess; ++p)
        if (!s->ev_plane[p]) e = cudaEventCreateWithFlags(&s->ev_plane[p], cudaEventDisableTiming);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
        if (!s->ev_join[j]) e = cudaEventCreateWithFlags(&s->ev_join[j], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (cudaStream_t h : es.st)
            if (h) cudaStreamDestroy(h);
        return e;
    }
    s->ev_streams.push_back(es);
    fs[0] = es.st[0];
    fs[1] = es.st[1];
    return cudaSuccess;
}

// run_event of a folded handle with several planes, stage timing off, on a stream above the
// device's lowest priority: each plane is rasterized on the caller's stream as before, and its
// convolution then runs on fork stream p mod 2 (each with its own spectrum scratch, at the
// caller's priority) while the caller's stream goes on with the next plane's raster; the
// caller's stream finally waits for both fork streams.  One plane's transforms thus overlap
// another's and the next raster, as in run_batch.  Work on the lowest-priority stream is
// background work and keeps the single-stream form: spread over three streams it holds more
// of the GPU at once, and higher-priority streams' work then waits longer for SMs (measured
// on a served mix: light-event p50 latency 0.85 -> 2-8 ms at 0.8-0.95 load when heavy
// low-priority events forked).  *taken = false (and nothing enqueued) when this form does
// not apply or its scratch cannot be had; the caller then runs the planes one after the other
// on its stream.
wct_status_t run_event_forked(wct_sim *s, const wct_depos_t *d, float *const *wfs, cudaStream_t cs, bool *taken) {
    *taken = false;
    if (s->timing || s->n_planes < 2 || s->ev_overlap_off) return WCT_OK;
    for (int p = 0; p < s->n_planes; ++p)
        if (s->planes[p].n_phases > 0) return WCT_OK;
    int prio = 0, lowest = 0, highest = 0;
    if (cudaStreamGetPriority(cs, &prio) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&lowest, &highest) != cudaSuccess) {
        cudaGetLastError();
        return WCT_OK;
    }
    if (prio >= lowest) return WCT_OK;                 // background work: one stream
    if (!s->bspec[1][0] || s->bspec_elems[1] < s->spec_elems) {
        // the second stream's spectra; without them (memory or budget) run_event stays serial
        const std::string keep = s->err;
        if (ensure_conv_spectra(s, 2) != WCT_OK) {
            s->err = keep;
            s->ev_overlap_off = true;
            return WCT_OK;
        }
    }
    cudaStream_t fs[2] = {};
    if (event_streams(s, cs, fs) != cudaSuccess) {
        cudaGetLastError();
        s->ev_overlap_off = true;
        return WCT_OK;
    }
    *taken = true;
    wct_status_t st = WCT_OK;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < s->n_planes && st == WCT_OK && e == cudaSuccess; ++p) {
        float *grid = s->grids[0] + s->grid_off[p];
        uint32_t *flags = s->tile_flags[0] + s->flag_off[p];
        const int j = p & 1;
        if ((st = raster_scatter(s, p, d, grid, cs, -1, false, flags))) break;
        e = cudaEventRecord(s->ev_plane[p], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs[j], s->ev_plane[p], 0);
        if (e == cudaSuccess) st = convolve_plane(s, p, grid, wfs[p], fs[j], -1, grid, flags, j);
    }
    // join, also after a failure, so that no forked work outlives the call unordered
    for (int j = 0; j < 2; ++j) {
        cudaError_t e2 = cudaEventRecord(s->ev_join[j], fs[j]);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(cs, s->ev_join[j], 0);
        if (e == cudaSuccess) e = e2;
    }
    if (st == WCT_OK && e != cudaSuccess) st = cuda_fail(s, e, "run_event streams");
    if (st) {
        cudaDeviceSynchronize();                       // forked work done before the grids are reset
        clear_grids(s);
    }
    return st;
}

}  // namespace

extern "C" {

wct_status_t wct_sim_create(const wct_plane_t *planes, int n_planes, const wct_response_t *responses,
                            const wct_diffusion_t *diffusion, const wct_opts_t *opts, wct_sim_t **out) {
    if (!out) return WCT_EINVAL;
    *out = nullptr;
    if (!planes || !responses || !diffusion || n_planes < 1 || n_planes > kMaxPlanes) return WCT_EINVAL;
    const wct_diffusion_t &df = *diffusion;
    if (!finite_pos(df.v_drift_mm_us) || !std::isfinite(df.DL_cm2_s) || df.DL_cm2_s < 0 ||
        !std::isfinite(df.DT_cm2_s) || df.DT_cm2_s < 0 || !finite_pos(df.nsigma))
        return WCT_EINVAL;
    for (int p = 0; p < n_planes; ++p) {
        const wct_plane_t &g = planes[p];
        const wct_response_t &r = responses[p];
        if (g.n_wires < 1 || g.n_ticks < 1 || g.n_impact_per_pitch < 1 || g.n_impact_per_pitch > 4096) return WCT_EINVAL;
        if (!finite_pos(g.pitch_mm) || !finite_pos(g.tick_us) || !std::isfinite(g.pitch_origin_mm) ||
            !std::isfinite(g.wire_angle_rad) || !std::isfinite(g.t_window0_us))
            return WCT_EINVAL;
        if ((int64_t)g.n_wires * g.n_ticks > ((int64_t)1 << 31)) return WCT_EINVAL;
        if (!r.host_data || r.n_wires_resp < 1 || (r.n_wires_resp & 1) == 0 ||
            r.n_wires_resp > WCT_MAX_RESPONSE_WIRES || r.n_ticks_resp < 1 || r.n_ticks_resp > 65536)
            return WCT_EINVAL;
    }
    wct_sim *s = new (std::nothrow) wct_sim();
    if (!s) return WCT_ENOMEM;
    cudaGetDevice(&s->device);
    s->n_planes = n_planes;
    s->diff = df;
    if (opts) {
        s->opts = *opts;
    } else {
        s->opts.hbm_budget_bytes = 0;
        s->opts.schedule_id = -1;
        s->opts.deterministic = 0;
    }
    // schedule_id: -1 default; otherwise bits 0, 2 and 3 = row transforms (0 register-staged,
    // 1 persistent bulk-copy, 4 persistent paired, 8 paired with composite radices), bit 1 =
    // rasterize (0 warp-level chunks, 1 CTA-level chunks).  Kept per handle, in its plans.
    int row_schedule = kDefaultRowSchedule, raster_schedule = 0;
    if (s->opts.schedule_id >= 0) {
        const int id = s->opts.schedule_id;
        row_schedule = (id & 8) ? 3 : (id & 4) ? 2 : (id & 1);
        raster_schedule = (id >> 1) & 1;
        // run_batch: bits 4-7 = v > 0 limit a persistent raster launch to 2^(v-1) events (chunks
        // that pipeline with the previous chunk's convolutions); bit 8 = one convolution stream
        const int v = (id >> 4) & 15;
        s->batch_events_per_launch = v > 0 ? 1 << (v - 1) : 0;
        s->conv_streams = ((id >> 8) & 1) ? 1 : ((id >> 9) & 1) ? 3 : 2;
    }
    s->det = s->opts.deterministic != 0;
    if (s->det) raster_schedule = 0;   // the fixed-point accumulation exists in the warp-level rasterizer
    wct_status_t st = WCT_OK;
    size_t spec_elems = 0;
    int max_tiles = 1;
    for (int p = 0; p < n_planes && st == WCT_OK; ++p) {
        PlaneState &ps = s->planes[p];
        ps.g = planes[p];
        const wct_plane_t &g = planes[p];
        PlaneParams &pp = ps.pp;
        pp.pitch = g.pitch_mm;
        pp.origin = g.pitch_origin_mm;
        pp.cos_a = std::cos(g.wire_angle_rad);
        pp.sin_a = std::sin(g.wire_angle_rad);
        pp.tick = g.tick_us;
        pp.tw0 = g.t_window0_us;
        pp.dp = g.pitch_mm / (double)g.n_impact_per_pitch;
        pp.DL = df.DL_cm2_s * 1.0e-4;   // cm^2/s -> mm^2/us
        pp.DT = df.DT_cm2_s * 1.0e-4;
        pp.v = df.v_drift_mm_us;
        pp.nsigma = df.nsigma;
        pp.inv_tick = 1.0 / g.tick_us;
        pp.inv_vtick = 1.0 / (df.v_drift_mm_us * g.tick_us);
        pp.inv_dp = 1.0 / pp.dp;
        {
            const double c[7] = {pp.inv_vtick, pp.inv_tick, pp.tw0, pp.cos_a, pp.sin_a, pp.origin, pp.inv_dp};
            for (int k = 0; k < 7; ++k) {
                pp.ff[k][0] = (float)c[k];
                pp.ff[k][1] = (float)(c[k] - (double)pp.ff[k][0]);
            }
        }
        // sigma_t = sqrt(2 D_L x / v) / v / tick, sigma_p = sqrt(2 D_T x / v) / dp
        pp.kt = (float)(std::sqrt(2.0 * pp.DL / df.v_drift_mm_us) / (df.v_drift_mm_us * g.tick_us));
        pp.kp = (float)(std::sqrt(2.0 * pp.DT / df.v_drift_mm_us) / pp.dp);
        pp.n_imp = g.n_impact_per_pitch;
        pp.n_wires = g.n_wires;
        pp.n_ticks = g.n_ticks;
        pp.plane_index = p;
        pp.fluctuate = df.fluctuate ? 1 : 0;
        pp.raster_schedule = raster_schedule;
        pp.key0 = (uint32_t)(df.seed & 0xFFFFFFFFu);
        pp.key1 = (uint32_t)(df.seed >> 32);
        for (int r = 0; r < 10; ++r) {   // round r uses key + r * (0x9E3779B9, 0xBB67AE85), mod 2^32
            pp.rk[2 * r] = pp.key0 + (uint32_t)r * 0x9E3779B9u;
            pp.rk[2 * r + 1] = pp.key1 + (uint32_t)r * 0xBB67AE85u;
        }
        pp.tile_w = tile_wires();
        pp.tile_t = tile_ticks();
        pp.n_tiles_w = (g.n_wires + pp.tile_w - 1) / pp.tile_w;
        pp.n_tiles_t = (g.n_ticks + pp.tile_t - 1) / pp.tile_t;
        ps.n_tiles = pp.n_tiles_w * pp.n_tiles_t;
        max_tiles = std::max(max_tiles, ps.n_tiles);
        const int max_wires = (WCT_MAX_WINDOW_IMPACTS - 1) / g.n_impact_per_pitch + 2;
        const int tw_max = (max_wires + pp.tile_w - 2) / pp.tile_w + 1;
        const int tt_max = (WCT_MAX_WINDOW_TICKS + pp.tile_t - 2) / pp.tile_t + 1;
        ps.max_tiles_per_depo = tw_max * tt_max;
        if (!plan_fft(g.n_ticks, responses[p].n_ticks_resp, ps.fft)) {
            st = fail(s, WCT_EINVAL, "no FFT plan for this tick count (too long)");
            break;
        }
        ps.fft.row_schedule = row_schedule;
        st = upload_twiddles(s, ps.fft);
    }
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->tile_count, sizeof(int32_t) * (max_tiles + 1));
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->tile_off, sizeof(int32_t) * (max_tiles + 1));
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->tile_cursor, sizeof(int32_t) * (max_tiles + 1));
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->scan32, sizeof(int32_t) * scan_tmp_elems(max_tiles + 1));
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->status, 4 * sizeof(int32_t));   // code + bounds record
    if (st == WCT_OK) {
        cudaError_t e = cudaMemset(s->status, 0, 4 * sizeof(int32_t));
        if (e != cudaSuccess) st = cuda_fail(s, e, "status init");
    }
    // Response spectra: pad each response to 21 centred rows, real-FFT the rows along ticks
    // with the same transform as the grid, and fold the inverse transform's 1/M into them.
    for (int p = 0; p < n_planes && st == WCT_OK; ++p) {
        PlaneState &ps = s->planes[p];
        const wct_response_t &r = responses[p];
        const int KW = WCT_MAX_RESPONSE_WIRES;
        const int off = (KW - r.n_wires_resp) / 2;
        std::vector<float> pad((size_t)KW * r.n_ticks_resp, 0.f);
        for (int row = 0; row < r.n_wires_resp; ++row)
            std::memcpy(&pad[(size_t)(row + off) * r.n_ticks_resp], r.host_data + (size_t)row * r.n_ticks_resp,
                        sizeof(float) * r.n_ticks_resp);
        float *d_resp = nullptr;
        st = dev_alloc(s, (void **)&d_resp, sizeof(float) * pad.size());
        if (st == WCT_OK) st = dev_alloc(s, (void **)&ps.resp_spec, sizeof(float2) * (size_t)KW * ps.fft.Fs);
        if (st != WCT_OK) break;
        cudaError_t e = cudaMemcpy(d_resp, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_row_r2c(ps.fft, d_resp, r.n_ticks_resp, r.n_ticks_resp, KW, ps.resp_spec, 0);
        if (e == cudaSuccess)
            e = launch_scale_spectrum(ps.resp_spec, (int64_t)KW * ps.fft.Fs, 1.0f / (float)ps.fft.M, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        dev_free(s, d_resp, sizeof(float) * pad.size());
        if (e != cudaSuccess) {
            st = cuda_fail(s, e, "response spectrum");
            break;
        }
        // Spectral support: the time spectra of the response rows decay fast (smooth field and
        // shaping functions).  Bins where every row's exact (FP64) spectrum is below FP32
        // machine epsilon (2^-23) times the largest magnitude are at the level of the rounding
        // of the FP32 response samples themselves; they are treated as zero, and only the bins
        // below the support go through the wire stage and the inverse transform.  A response
        // with full support (e.g. a delta) keeps every bin.
        std::vector<float2> hs((size_t)KW * ps.fft.Fs);
        e = cudaMemcpy(hs.data(), ps.resp_spec, sizeof(float2) * hs.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = cuda_fail(s, e, "response spectrum support");
            break;
        }
        double gmax = 0.0;   // scale of the threshold from the device spectrum (FP32-accurate)
        for (int k = 0; k < KW; ++k)
            for (int f = 0; f < ps.fft.F; ++f) {
                const float2 v = hs[(size_t)k * ps.fft.Fs + f];
                gmax = std::max(gmax, std::sqrt((double)v.x * v.x + (double)v.y * v.y));
            }
        const int last = response_support_last(r, 2 * ps.fft.M, ps.fft.F, 0x1p-23 * gmax * (double)ps.fft.M);
        const int Fu = std::min(ps.fft.Fs, (last + 2) & ~1);
        if (Fu < ps.fft.Fs) {
            // the grid spectra and the response spectrum keep only the supported bins: row
            // stride Fu (even, so rows stay 16-byte aligned)
            float2 *packed = nullptr;
            st = dev_alloc(s, (void **)&packed, sizeof(float2) * (size_t)KW * Fu);
            if (st != WCT_OK) break;
            e = cudaMemcpy2D(packed, sizeof(float2) * Fu, ps.resp_spec, sizeof(float2) * ps.fft.Fs, sizeof(float2) * Fu,
                             KW, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) {
                st = cuda_fail(s, e, "response spectrum support");
                break;
            }
            dev_free(s, ps.resp_spec, sizeof(float2) * (size_t)KW * ps.fft.Fs);
            ps.resp_spec = packed;
            ps.fft.Fs = Fu;
        }
        ps.fft.Fu = Fu;
        spec_elems = std::max(spec_elems, (size_t)ps.g.n_wires * ps.fft.Fs);
    }
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->spec, sizeof(float2) * spec_elems);
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->spec2, sizeof(float2) * spec_elems);
    s->spec_elems = spec_elems;
    for (int p = 0; p < n_planes; ++p) s->max_wires = std::max(s->max_wires, s->planes[p].g.n_wires);
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->act[0][0], 2 * (size_t)s->max_wires);
    if (st == WCT_OK) s->act[0][1] = s->act[0][0] + s->max_wires;
    for (int p = 0; p < n_planes; ++p) {
        s->grid_off[p + 1] = s->grid_off[p] + (size_t)s->planes[p].g.n_wires * s->planes[p].g.n_ticks;
        s->flag_off[p + 1] = s->flag_off[p] + tile_flag_words(s->planes[p].pp);
    }
    if (st == WCT_OK && s->det) {
        st = dev_alloc(s, (void **)&s->det_flags, sizeof(uint32_t) * s->flag_off[n_planes]);
        if (st == WCT_OK && cudaMemset(s->det_flags, 0, sizeof(uint32_t) * s->flag_off[n_planes]))
            st = fail(s, WCT_ECUDA, "grid init");
    }
    if (st == WCT_OK) st = dev_alloc(s, (void **)&s->work_counter, sizeof(unsigned long long));
    if (st == WCT_OK) st = add_grid_set(s);   // set 0: run_event's
    if (st != WCT_OK) {
        for (auto &a : s->allocs)
            if (a.first) cudaFree(a.first);
        delete s;
        return st;
    }
    *out = s;
    return WCT_OK;
}

wct_status_t wct_sim_destroy(wct_sim_t *s) {
    if (!s) return WCT_EINVAL;
    cudaDeviceSynchronize();
    for (auto &a : s->allocs)
        if (a.first) cudaFree(a.first);
    for (auto &slot : s->slots)
        for (auto &e : slot) cudaEventDestroy(e);
    for (auto &slot : s->bslots)
        for (auto &e : slot) cudaEventDestroy(e);
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    for (cudaStream_t h : {s->rs_stream, s->cv_stream[0], s->cv_stream[1], s->cv_stream[2]})
        if (h) cudaStreamDestroy(h);
    for (auto &e : s->evpool)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t h : {s->up_stream, s->comp_stream, s->down_stream})
        if (h) cudaStreamDestroy(h);
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t h : {s->ev_up[b], s->ev_comp[b], s->ev_down[b]})
            if (h) cudaEventDestroy(h);
    for (auto &es : s->ev_streams)
        for (cudaStream_t h : es.st)
            if (h) cudaStreamDestroy(h);
    for (cudaEvent_t h : s->ev_plane)
        if (h) cudaEventDestroy(h);
    for (cudaEvent_t h : s->ev_join)
        if (h) cudaEventDestroy(h);
    delete s;
    return WCT_OK;
}

wct_status_t wct_sim_rasterize(wct_sim_t *s, int plane, const wct_depos_t *d, float *patches, int64_t capacity,
                               int64_t *patch_desc, int64_t *total_bins, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if ((st = check_depos(s, d))) return st;
    if (!patch_desc || !total_bins) return fail(s, WCT_EINVAL, "patch_desc and total_bins are required");
    cudaStream_t cs = (cudaStream_t)stream;
    if ((st = ensure_depo_capacity(s, d->n))) return st;
    const PlaneParams pp = plane_params(s, plane);
    cudaError_t e = launch_prep(*d, pp, s->desc, nullptr, s->patch_size, s->status, cs);
    if (e == cudaSuccess) e = launch_scan_i64(s->patch_size, s->patch_off, d->n, s->scan64, cs);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, s->patch_off + d->n, sizeof(int64_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(s, e, "rasterize sizing");
    *total_bins = total;
    const bool write = patches && total <= capacity;
    e = launch_rasterize_patches(d->n, s->desc, s->patch_off, pp, (uint32_t)d->event_id, write ? patches : nullptr,
                                 patch_desc, cs);
    if (e != cudaSuccess) return cuda_fail(s, e, "rasterize");
    s->launches += (d->n > 0 ? 3 : 0) + 3 + (write && d->n > 0 ? 1 : 0);
    if (patches && !write) return fail(s, WCT_EINVAL, "patch buffer smaller than total_bins");
    return WCT_OK;
}

wct_status_t wct_sim_rasterize_fixed(wct_sim_t *s, int plane, const wct_depos_t *d, float *patches, int64_t slot_bins,
                                     int64_t *patch_desc, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if ((st = check_depos(s, d))) return st;
    if (!patches || !patch_desc) return fail(s, WCT_EINVAL, "patches and patch_desc are required");
    if (slot_bins < 1 || slot_bins > (int64_t)WCT_MAX_WINDOW_TICKS * WCT_MAX_WINDOW_IMPACTS)
        return fail(s, WCT_EINVAL, "slot_bins out of range");
    cudaStream_t cs = (cudaStream_t)stream;
    if ((st = ensure_depo_capacity(s, d->n))) return st;
    const PlaneParams pp = plane_params(s, plane);
    cudaError_t e = launch_prep(*d, pp, s->desc, nullptr, s->patch_size, s->status, cs);
    if (e == cudaSuccess) e = launch_fit_slots(d->n, s->desc, slot_bins, s->status, cs);
    if (e == cudaSuccess)
        e = launch_rasterize_patches(d->n, s->desc, nullptr, pp, (uint32_t)d->event_id, patches, patch_desc, cs, slot_bins);
    if (e != cudaSuccess) return cuda_fail(s, e, "rasterize fixed");
    s->launches += d->n > 0 ? 4 : 0;
    return WCT_OK;
}

wct_status_t wct_sim_patch_slot_bins(wct_sim_t *s, int plane, double x_max_mm, int64_t *slot_bins) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if (!slot_bins) return fail(s, WCT_EINVAL, "slot_bins is NULL");
    if (!std::isfinite(x_max_mm) || x_max_mm < 0.0) return fail(s, WCT_EINVAL, "x_max_mm must be finite and >= 0");
    // the widths as depo_window_f64 forms them (sigma grows with the drift distance, so the
    // widest windows are those at x_max), then the window rule: the bins overlapping
    // [mu - n sigma, mu + n sigma] number floor(mu + n sigma) - floor(mu - n sigma) + 1, at most
    // floor(2 n sigma) + 2 over every position mu; a point charge (sigma < 1e-6 bin) takes one bin
    const PlaneParams &pp = s->planes[plane].pp;
    const double td = x_max_mm / pp.v;
    const double s_t = std::sqrt((2.0 * pp.DL) * td) / pp.v / pp.tick;
    const double s_p = std::sqrt((2.0 * pp.DT) * td) / pp.dp;
    auto extent = [&](double sg, int64_t cap) -> int64_t {
        if (sg < 1e-6) return 1;
        const double e = std::floor(2.0 * (pp.nsigma * sg)) + 2.0;
        return e < (double)cap ? (int64_t)e : cap;   // a wider window is an invalid depo, never rasterized
    };
    *slot_bins = extent(s_t, WCT_MAX_WINDOW_TICKS) * extent(s_p, WCT_MAX_WINDOW_IMPACTS);
    return WCT_OK;
}

wct_status_t wct_sim_scatter(wct_sim_t *s, int plane, const wct_depos_t *d, const float *patches,
                             const int64_t *patch_desc, float *grid, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if ((st = check_depos(s, d))) return st;
    if (!grid) return fail(s, WCT_EINVAL, "grid is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    if ((st = ensure_depo_capacity(s, d->n))) return st;
    if (!patches) return raster_scatter(s, plane, d, grid, cs, -1);
    if (!patch_desc) return fail(s, WCT_EINVAL, "patch_desc is required with patches");
    const PlaneState &ps = s->planes[plane];
    const PlaneParams pp = plane_params(s, plane);
    cudaError_t e = cudaMemsetAsync(s->tile_count, 0, sizeof(int32_t) * (ps.n_tiles + 1), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->tile_cursor, 0, sizeof(int32_t) * (ps.n_tiles + 1), cs);
    if (e == cudaSuccess) e = launch_bin_patches(d->n, patch_desc, pp, s->tile_count, s->status, cs);
    if (e == cudaSuccess) e = launch_scan_i32(s->tile_count, s->tile_off, ps.n_tiles, s->scan32, cs);
    if (e == cudaSuccess)
        e = launch_fill_patches(d->n, patch_desc, pp, s->tile_off, s->tile_cursor, s->tile_list, s->list_cap,
                                s->status, cs);
    if (e == cudaSuccess)
        e = launch_tile_scatter_patches(patch_desc, patches, s->tile_off, s->tile_list, s->list_cap, pp, grid, cs, s->det,
                                        s->status);
    if (e != cudaSuccess) return cuda_fail(s, e, "scatter patches");
    s->launches += 4 + (d->n > 0 ? 2 : 0);
    return WCT_OK;
}

wct_status_t wct_sim_convolve(wct_sim_t *s, int plane, const float *grid, float *wf, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if (!grid || !wf) return fail(s, WCT_EINVAL, "grid / waveform is NULL");
    return convolve_plane(s, plane, grid, wf, (cudaStream_t)stream, -1);
}

wct_status_t wct_sim_run_event(wct_sim_t *s, const wct_depos_t *d, float *const *wfs, void *stream) {
    if (!s) return WCT_EINVAL;
    wct_status_t st = check_depos(s, d);
    if (st) return st;
    if (!wfs) return fail(s, WCT_EINVAL, "waveforms is NULL");
    for (int p = 0; p < s->n_planes; ++p)
        if (!wfs[p]) return fail(s, WCT_EINVAL, "a waveform pointer is NULL");
    if ((st = ensure_depo_capacity(s, d->n))) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    bool taken = false;
    st = run_event_forked(s, d, wfs, cs, &taken);
    if (taken) return st;
    for (int p = 0; p < s->n_planes; ++p) {
        // accumulate into the library grid (all zero), which the forward transform clears
        // again as it reads it; the inverse transform writes the caller's waveform
        if (s->planes[p].n_phases > 0) {
            if ((st = run_plane_impact(s, p, d, wfs[p], cs, acquire_slot(s)))) {
                clear_grids(s);
                return st;
            }
            continue;
        }
        float *grid = s->grids[0] + s->grid_off[p];
        uint32_t *flags = s->tile_flags[0] + s->flag_off[p];
        const int slot = acquire_slot(s);
        mark(s, slot, 0, cs);
        if ((st = raster_scatter(s, p, d, grid, cs, slot, false, flags)) ||
            (st = convolve_plane(s, p, grid, wfs[p], cs, slot, grid, flags))) {
            clear_grids(s);
            return st;
        }
    }
    if (s->timing) ++s->events_timed;
    return WCT_OK;
}

}  // extern "C"

namespace {

constexpr size_t kMaxGraphs = 8;

// run_batch.  The whole batch (or, under a memory limit or a schedule asking for it, a chunk of
// its events) is rasterized and scattered by ONE persistent launch over every (event, plane)
// pair, each event into a grid set of its own, on a library raster stream; the convolutions of
// the rasterized grids follow on library convolution streams (two by default, taking the
// (event, plane) pairs alternately, so one plane's transform overlaps the tail of another's),
// each with its own spectrum scratch.  With several chunks, the raster of chunk c + 1 overlaps
// the convolutions of chunk c.  All streams fork from and join back into the caller's stream.
wct_status_t batch_streams(wct_sim *s, cudaStream_t caller) {
    if (s->rs_stream) return WCT_OK;
    // the rasterize stream takes the priority of the stream of the first run_batch call and the
    // convolution streams the next higher one, so the convolution's CTAs go first whenever SMs
    // free up and the rasterize CTAs fill the remaining room, and a caller can rank one
    // handle's batches above another's (lower numbers run first)
    int lo = 0, hi = 0, own = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess && cudaStreamGetPriority(caller, &own) != cudaSuccess) {
        cudaGetLastError();
        own = lo;
    }
    own = std::min(std::max(own, hi), lo);
    const int conv = std::max(hi, own - 1);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->rs_stream, cudaStreamNonBlocking, own);
    for (int j = 0; j < 3 && e == cudaSuccess; ++j)
        e = cudaStreamCreateWithPriority(&s->cv_stream[j], cudaStreamNonBlocking, conv);
    if (e != cudaSuccess) return cuda_fail(s, e, "batch streams");
    return WCT_OK;
}

// The i-th event of the batch's event pool (created on first use; reused by later calls, whose
// records and waits are stream-ordered after this call's).
wct_status_t pool_event(wct_sim *s, size_t i, cudaEvent_t *out) {
    while (s->evpool.size() <= i) {
        cudaEvent_t e = nullptr;
        const cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (err != cudaSuccess) return cuda_fail(s, err, "batch events");
        s->evpool.push_back(e);
    }
    *out = s->evpool[i];
    return WCT_OK;
}

// Batch grid sets 1..want (set 0 is run_event's); stops early when memory runs out, as long as
// at least one batch set exists.  *have receives the number of batch sets.
wct_status_t ensure_batch_sets(wct_sim *s, int want, int *have) {
    while ((int)s->grids.size() < want + 1) {
        const wct_status_t st = add_grid_set(s);
        if (st == WCT_ENOMEM && s->grids.size() > 1) {
            s->err.clear();
            break;
        }
        if (st) return st;
    }
    *have = std::min(want, (int)s->grids.size() - 1);
    return WCT_OK;
}

// The spectrum scratch of convolution streams 1 .. n - 1, as large as stream 0's (spec, spec2).
wct_status_t ensure_conv_spectra(wct_sim *s, int n) {
    for (int j = 1; j < n; ++j) {
        if (s->bspec[j][0] && s->bspec_elems[j] >= s->spec_elems) continue;
        dev_free(s, s->bspec[j][0]);
        dev_free(s, s->bspec[j][1]);
        s->bspec[j][0] = s->bspec[j][1] = nullptr;
        s->bspec_elems[j] = 0;
        dev_free(s, s->act[j][0]);
        s->act[j][0] = s->act[j][1] = nullptr;
        const wct_status_t st = dev_alloc_all(s, {{(void **)&s->bspec[j][0], sizeof(float2) * s->spec_elems},
                                                  {(void **)&s->bspec[j][1], sizeof(float2) * s->spec_elems},
                                                  {(void **)&s->act[j][0], 2 * (size_t)s->max_wires}});
        if (st) return st;
        s->act[j][1] = s->act[j][0] + s->max_wires;
        s->bspec_elems[j] = s->spec_elems;
    }
    return WCT_OK;
}

wct_status_t enqueue_batch(wct_sim *s, const wct_depos_t *events, int n_events, float *const *wfs, cudaStream_t st) {
    wct_status_t r = batch_streams(s, st);
    if (r) return r;
    const int npl = s->n_planes;
    // events per raster launch: the whole batch unless the schedule asks for smaller chunks; a
    // launch's table holds at most kBatchItems (event, plane) pairs
    int per = s->batch_events_per_launch > 0 ? s->batch_events_per_launch : n_events;
    per = std::max(1, std::min({per, n_events, kBatchItems / npl}));
    int n_chunks = (n_events + per - 1) / per;
    // grid sets: one per event of a launch, twice that when chunks alternate (so the raster of
    // chunk c + 1 never waits for the convolutions of chunk c)
    int have = 0;
    if ((r = ensure_batch_sets(s, n_chunks > 1 ? 2 * per : per, &have))) return r;
    if (have < (n_chunks > 1 ? 2 * per : per)) {
        per = std::max(1, have >= 2 ? have / 2 : 1);
        n_chunks = (n_events + per - 1) / per;
    }
    const bool alternate = n_chunks > 1 && have >= 2 * per;
    const int nc = std::max(1, std::min(3, s->conv_streams));
    if ((r = ensure_conv_spectra(s, nc))) return r;
    // largest events first: the persistent launch hands out their chunks before the small ones'
    std::vector<int> order(n_events);
    for (int e = 0; e < n_events; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return events[a].n > events[b].n; });
    static thread_local BatchTable tab;   // ~25 KB: kept off the stack
    for (int p = 0; p < npl; ++p) tab.plane[p] = s->planes[p].pp;
    cudaStream_t rs = s->rs_stream, *cv = s->cv_stream;
    // events of the pool: 0 fork, then per chunk c: 1 + 4c raster done, 2 + 4c + j its
    // convolutions done on convolution stream j
    cudaEvent_t fork = nullptr;
    if ((r = pool_event(s, 0, &fork))) return r;
    cudaError_t err = cudaEventRecord(fork, st);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(rs, fork, 0);
    for (int j = 0; j < nc && err == cudaSuccess; ++j) err = cudaStreamWaitEvent(cv[j], fork, 0);
    if (err != cudaSuccess) return cuda_fail(s, err, "batch fork");
    int k_conv = 0;   // (event, plane) pairs convolved so far: they take the streams in turn
    for (int c = 0; c < n_chunks; ++c) {
        const int e0 = c * per, e1 = std::min(n_events, e0 + per);
        const int base = 1 + (alternate ? (c & 1) * per : 0);   // first grid set of this chunk
        cudaEvent_t rdone = nullptr, cdone[3] = {};
        if ((r = pool_event(s, 1 + 4 * (size_t)c, &rdone))) return r;
        for (int j = 0; j < nc; ++j)
            if ((r = pool_event(s, 2 + 4 * (size_t)c + j, &cdone[j]))) return r;
        // the sets were last used by chunk c - 2 (alternating) or c - 1: wait for their clearing
        const int prev = alternate ? c - 2 : c - 1;
        if (prev >= 0)
            for (int j = 0; j < nc && err == cudaSuccess; ++j) err = cudaStreamWaitEvent(rs, s->evpool[2 + 4 * prev + j], 0);
        if (err != cudaSuccess) return cuda_fail(s, err, "batch grid dependency");
        int64_t chunks = 0;
        tab.n_items = 0;
        for (int i = e0; i < e1; ++i) {
            const wct_depos_t &d = events[order[i]];
            if (d.n <= 0) continue;
            const int set = base + (i - e0);
            for (int p = 0; p < npl; ++p) {
                BatchItem &b = tab.item[tab.n_items++];
                b.t0 = d.t0_us;
                b.x = d.x_mm;
                b.y = d.y_mm;
                b.z = d.z_mm;
                b.q = d.q_e;
                b.n = d.n;
                b.grid = s->grids[set] + s->grid_off[p];
                b.grid64 = s->det ? s->grids64[set] + s->grid_off[p] : nullptr;
                b.flags = s->tile_flags[set] + s->flag_off[p];
                b.chunk_begin = chunks;
                b.event_lo = (uint32_t)d.event_id;
                b.plane = p;
                chunks += raster_chunk_count(d.n, 0);
            }
        }
        const int tslot = acquire_batch_slot(s);
        bmark(s, tslot, 0, rs);
        if (chunks > 0) {
            err = launch_raster_batch_persistent(tab, chunks, s->work_counter, s->status, rs, s->det);
            if (err != cudaSuccess) return cuda_fail(s, err, "batched raster-scatter");
            s->launches += 1;
        }
        bmark(s, tslot, 1, rs);
        err = cudaEventRecord(rdone, rs);
        for (int j = 0; j < nc && err == cudaSuccess; ++j) err = cudaStreamWaitEvent(cv[j], rdone, 0);
        if (err != cudaSuccess) return cuda_fail(s, err, "batch dependency");
        bmark(s, tslot, 2, cv[0]);
        bmark(s, tslot, 4, cv[nc - 1]);
        for (int i = e0; i < e1; ++i) {
            const int e = order[i], set = base + (i - e0);
            for (int p = 0; p < npl; ++p, ++k_conv) {
                const int j = k_conv % nc;
                float *grid = s->grids[set] + s->grid_off[p];
                if (s->det && events[e].n > 0) {
                    // deterministic mode: the touched fixed-point tiles into the float grid, on
                    // the stream that convolves it (overlapping the other stream's work)
                    const PlaneParams &pp = s->planes[p].pp;
                    err = launch_fix_tiles(s->tile_flags[set] + s->flag_off[p], pp.n_wires, pp.n_ticks, pp.tile_w,
                                           pp.tile_t, s->grids64[set] + s->grid_off[p], grid, cv[j], s->status);
                    if (err != cudaSuccess) return cuda_fail(s, err, "fixed-point grid");
                    s->launches += 1;
                }
                r = convolve_plane(s, p, grid, wfs[(size_t)e * npl + p], cv[j], -1, grid,
                                   s->tile_flags[set] + s->flag_off[p], j);
                if (r) return r;
            }
        }
        bmark(s, tslot, 3, cv[0]);
        bmark(s, tslot, 5, cv[nc - 1]);
        for (int j = 0; j < nc && err == cudaSuccess; ++j) err = cudaEventRecord(cdone[j], cv[j]);
        if (err != cudaSuccess) return cuda_fail(s, err, "batch grid dependency");
    }
    if (s->timing) ++s->batches_timed;
    // join: the caller's stream waits for the last chunk's convolutions and the raster stream
    const int last = n_chunks - 1;
    err = cudaSuccess;
    for (int j = 0; j < nc && err == cudaSuccess; ++j) err = cudaStreamWaitEvent(st, s->evpool[2 + 4 * last + j], 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, s->evpool[1 + 4 * last], 0);
    if (err != cudaSuccess) return cuda_fail(s, err, "batch join");
    return WCT_OK;
}

}  // namespace

extern "C" {

wct_status_t wct_sim_run_batch(wct_sim_t *s, const wct_depos_t *events, int n_events, float *const *wfs,
                               void *stream) {
    if (!s) return WCT_EINVAL;
    if (n_events < 0 || (n_events > 0 && (!events || !wfs))) return fail(s, WCT_EINVAL, "bad batch arguments");
    for (int e = 0; e < n_events; ++e) {
        wct_status_t st = check_depos(s, &events[e]);
        if (st) return st;
        for (int p = 0; p < s->n_planes; ++p)
            if (!wfs[(size_t)e * s->n_planes + p]) return fail(s, WCT_EINVAL, "a waveform pointer is NULL");
    }
    if (n_events == 0) return WCT_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    for (int p = 0; p < s->n_planes; ++p)
        if (s->planes[p].n_phases > 0) {
            // impact mode: events one after the other (no batched rasterize launch)
            for (int e = 0; e < n_events; ++e) {
                const wct_status_t st = wct_sim_run_event(s, &events[e], wfs + (size_t)e * s->n_planes, stream);
                if (st) return st;
            }
            return WCT_OK;
        }
    if (s->timing) return enqueue_batch(s, events, n_events, wfs, cs);   // timing events: no graph
    // graph key: everything the recorded launches depend on
    std::vector<uint64_t> key;
    key.reserve((size_t)n_events * (7 + s->n_planes) + 1);
    key.push_back((uint64_t)n_events);
    for (int e = 0; e < n_events; ++e) {
        const wct_depos_t &d = events[e];
        for (const void *ptr : {(const void *)d.t0_us, (const void *)d.x_mm, (const void *)d.y_mm,
                                (const void *)d.z_mm, (const void *)d.q_e})
            key.push_back((uint64_t)(uintptr_t)ptr);
        key.push_back((uint64_t)d.n);
        key.push_back(d.event_id);
        for (int p = 0; p < s->n_planes; ++p) key.push_back((uint64_t)(uintptr_t)wfs[(size_t)e * s->n_planes + p]);
    }
    for (auto &g : s->graphs) {
        if (g.key == key) {
            cudaError_t e = cudaGraphLaunch(g.exec, cs);
            if (e != cudaSuccess) return cuda_fail(s, e, "graph launch");
            ++s->graph_launches;
            s->launches += g.kernels;
            return WCT_OK;
        }
    }
    // record a graph only for a batch seen before: one-off batches launch directly
    auto it = std::find(s->seen.begin(), s->seen.end(), key);
    if (it == s->seen.end()) {
        if (s->seen.size() >= kMaxGraphs) s->seen.erase(s->seen.begin());
        s->seen.push_back(key);
        return enqueue_batch(s, events, n_events, wfs, cs);
    }
    s->seen.erase(it);
    if (!s->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(s, e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return enqueue_batch(s, events, n_events, wfs, cs);   // no graph: launch directly
    }
    const int64_t launches0 = s->launches;
    wct_status_t st = enqueue_batch(s, events, n_events, wfs, s->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s->cap_stream, &graph);
    if (st != WCT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        s->launches = launches0;
        if (st != WCT_OK) return st;
        return enqueue_batch(s, events, n_events, wfs, cs);
    }
    const int64_t recorded = s->launches - launches0;
    s->launches = launches0;   // counted when the graph runs
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->launches = launches0;
        return enqueue_batch(s, events, n_events, wfs, cs);
    }
    if (s->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(s->graphs.front().exec);
        s->graphs.erase(s->graphs.begin());
    }
    s->graphs.push_back({std::move(key), exec, recorded});
    e = cudaGraphLaunch(exec, cs);
    if (e != cudaSuccess) return cuda_fail(s, e, "graph launch");
    ++s->graph_launches;
    s->launches += recorded;
    return WCT_OK;
}

wct_status_t wct_sim_run_host(wct_sim_t *s, const wct_host_depos_t *events, int n_events, float *const *wfs) {
    if (!s || n_events < 0) return WCT_EINVAL;
    if (n_events == 0) return WCT_OK;
    if (!events || !wfs) return fail(s, WCT_EINVAL, "events or waveforms is NULL");
    const int npl = s->n_planes;
    int64_t max_n = 1;
    for (int e = 0; e < n_events; ++e) {
        const wct_host_depos_t &h = events[e];
        if (h.n < 0 || h.n > ((int64_t)1 << 30)) return fail(s, WCT_EINVAL, "bad depo count");
        if (h.n > 0 && (!h.t0_us || !h.x_mm || !h.y_mm || !h.z_mm || !h.q_e))
            return fail(s, WCT_EINVAL, "a depo array pointer is NULL");
        for (int p = 0; p < npl; ++p)
            if (!wfs[(size_t)e * npl + p]) return fail(s, WCT_EINVAL, "a waveform pointer is NULL");
        max_n = std::max(max_n, h.n);
    }
    // the pipeline runs on the library's own streams: wait for work already enqueued on the
    // device (this handle's earlier calls on any stream share its scratch)
    cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) return cuda_fail(s, err, "host pipeline: earlier work");
    if (!s->up_stream) {
        for (cudaStream_t *h : {&s->up_stream, &s->comp_stream, &s->down_stream})
            if (err == cudaSuccess) err = cudaStreamCreateWithFlags(h, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b)
            for (cudaEvent_t *h : {&s->ev_up[b], &s->ev_comp[b], &s->ev_down[b]})
                if (err == cudaSuccess) err = cudaEventCreateWithFlags(h, cudaEventDisableTiming);
        if (err != cudaSuccess) return cuda_fail(s, err, "host pipeline streams");
    }
    wct_status_t st = WCT_OK;
    if (!s->h_wave[0][0]) {
        // all staging waveforms or none (a failed first call leaves nothing half-allocated)
        for (int b = 0; b < 2 && st == WCT_OK; ++b)
            for (int p = 0; p < npl && st == WCT_OK; ++p)
                st = dev_alloc(s, (void **)&s->h_wave[b][p],
                               sizeof(float) * (size_t)s->planes[p].g.n_wires * s->planes[p].g.n_ticks);
        if (st) {
            for (int b = 0; b < 2; ++b)
                for (int p = 0; p < npl; ++p) {
                    dev_free(s, s->h_wave[b][p]);
                    s->h_wave[b][p] = nullptr;
                }
            return st;
        }
    }
    if (max_n > s->h_cap) {
        // earlier calls returned only after their streams drained: the old staging is idle
        for (int b = 0; b < 2; ++b) {
            dev_free(s, s->h_depo[b]);
            s->h_depo[b] = nullptr;
        }
        s->h_cap = 0;
        st = dev_alloc_all(s, {{(void **)&s->h_depo[0], sizeof(float) * 5 * (size_t)max_n},
                               {(void **)&s->h_depo[1], sizeof(float) * 5 * (size_t)max_n}});
        if (st) return st;
        s->h_cap = max_n;
    }
    cudaStream_t up = s->up_stream, comp = s->comp_stream, down = s->down_stream;
    for (int e = 0; e < n_events && st == WCT_OK && err == cudaSuccess; ++e) {
        const int b = e & 1;
        const wct_host_depos_t &h = events[e];
        float *db = s->h_depo[b];
        const int64_t cap = s->h_cap;
        wct_depos_t d{db, db + cap, db + 2 * cap, db + 3 * cap, db + 4 * cap, h.n, h.event_id};
        // upload once the compute of event e - 2 has released this staging buffer
        if (e >= 2) err = cudaStreamWaitEvent(up, s->ev_comp[b], 0);
        const float *src[5] = {h.t0_us, h.x_mm, h.y_mm, h.z_mm, h.q_e};
        for (int a = 0; a < 5 && err == cudaSuccess && h.n > 0; ++a)
            err = cudaMemcpyAsync(db + a * cap, src[a], sizeof(float) * (size_t)h.n, cudaMemcpyHostToDevice, up);
        if (err == cudaSuccess) err = cudaEventRecord(s->ev_up[b], up);
        // compute once the upload landed and the download of event e - 2 freed the waveforms
        if (err == cudaSuccess) err = cudaStreamWaitEvent(comp, s->ev_up[b], 0);
        if (err == cudaSuccess && e >= 2) err = cudaStreamWaitEvent(comp, s->ev_down[b], 0);
        if (err != cudaSuccess) break;
        st = wct_sim_run_event(s, &d, s->h_wave[b], comp);
        if (st) break;
        err = cudaEventRecord(s->ev_comp[b], comp);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(down, s->ev_comp[b], 0);
        for (int p = 0; p < npl && err == cudaSuccess; ++p)
            err = cudaMemcpyAsync(wfs[(size_t)e * npl + p], s->h_wave[b][p],
                                  sizeof(float) * (size_t)s->planes[p].g.n_wires * s->planes[p].g.n_ticks,
                                  cudaMemcpyDeviceToHost, down);
        if (err == cudaSuccess) err = cudaEventRecord(s->ev_down[b], down);
    }
    // drain every stream before returning (also after an error: nothing may still use the staging)
    for (cudaStream_t h : {up, comp, down}) {
        const cudaError_t e2 = cudaStreamSynchronize(h);
        if (err == cudaSuccess) err = e2;
    }
    if (st) return st;   // run_event restored the grids
    if (err != cudaSuccess) {
        clear_grids(s);
        return cuda_fail(s, err, "host pipeline");
    }
    return wct_sim_sync(s, comp);
}

wct_status_t wct_sim_set_impact_responses(wct_sim_t *s, int plane, const wct_response_t *responses, int n_phases) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    PlaneState &ps = s->planes[plane];
    cudaDeviceSynchronize();                           // nothing may still use the old state
    drop_impact(s, ps);
    if (!responses) return WCT_OK;                     // back to the folded mode
    if (n_phases != ps.g.n_impact_per_pitch) return fail(s, WCT_EINVAL, "n_phases must equal n_impact_per_pitch");
    int kt = 0;
    for (int ph = 0; ph < n_phases; ++ph) {
        const wct_response_t &r = responses[ph];
        if (!r.host_data || r.n_wires_resp < 1 || (r.n_wires_resp & 1) == 0 || r.n_wires_resp > WCT_MAX_RESPONSE_WIRES ||
            r.n_ticks_resp < 1 || r.n_ticks_resp > 65536 || (ph > 0 && r.n_ticks_resp != kt))
            return fail(s, WCT_EINVAL, "bad impact response (odd wire extent <= 21, equal tick extents)");
        kt = r.n_ticks_resp;
    }
    FFTPlan full{};
    if (!plan_fft(ps.g.n_ticks, kt, full)) return fail(s, WCT_EINVAL, "no FFT plan for this tick count (too long)");
    full.tw = ps.fft.tw;                               // same transform length as the plane's
    full.rtw = ps.fft.rtw;
    full.row_schedule = ps.fft.row_schedule;
    if (full.M != ps.fft.M) return fail(s, WCT_EINVAL, "impact responses need the plane's transform length");
    // spectra of every phase, the common support, then one packed buffer
    const int KW = WCT_MAX_RESPONSE_WIRES;
    std::vector<float2 *> dspec(n_phases, nullptr);
    std::vector<std::vector<float2>> host(n_phases);
    double gmax = 0.0;
    for (int ph = 0; ph < n_phases && st == WCT_OK; ++ph) {
        st = response_spectrum(s, full, responses[ph], &dspec[ph], host[ph]);
        if (st == WCT_OK) gmax = std::max(gmax, spectrum_max(host[ph], full));
    }
    int last = 0;
    for (int ph = 0; ph < n_phases && st == WCT_OK; ++ph)
        last = std::max(last, response_support_last(responses[ph], 2 * full.M, full.F, 0x1p-23 * gmax * (double)full.M));
    const int Fu = std::min(full.Fs, (last + 2) & ~1);
    if (st == WCT_OK) {
        ps.resp_imp_bytes = sizeof(float2) * (size_t)n_phases * KW * Fu;
        st = dev_alloc(s, (void **)&ps.resp_imp, ps.resp_imp_bytes);
    }
    for (int ph = 0; ph < n_phases && st == WCT_OK; ++ph) {
        const cudaError_t e = cudaMemcpy2D(ps.resp_imp + (size_t)ph * KW * Fu, sizeof(float2) * Fu, dspec[ph],
                                           sizeof(float2) * full.Fs, sizeof(float2) * Fu, KW, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) st = cuda_fail(s, e, "impact response spectra");
    }
    for (int ph = 0; ph < n_phases; ++ph) dev_free(s, dspec[ph], sizeof(float2) * (size_t)KW * full.Fs);
    ps.fft_imp = full;
    ps.fft_imp.Fs = ps.fft_imp.Fu = Fu;
    // spectrum scratch must hold n_wires x Fu
    const size_t need = (size_t)ps.g.n_wires * Fu;
    if (st == WCT_OK && need > s->spec_elems) {
        // the folded mode keeps using the old scratch if the larger one cannot be had
        float2 *a = nullptr, *b = nullptr;
        st = dev_alloc_all(s, {{(void **)&a, sizeof(float2) * need}, {(void **)&b, sizeof(float2) * need}});
        if (st == WCT_OK) {
            dev_free(s, s->spec);
            dev_free(s, s->spec2);
            s->spec = a;
            s->spec2 = b;
            s->spec_elems = need;
        }
    }
    if (st == WCT_OK) {
        ps.phase_grid_bytes = sizeof(float) * (size_t)n_phases * ps.g.n_wires * ps.g.n_ticks;
        st = dev_alloc(s, (void **)&ps.phase_grids, ps.phase_grid_bytes);
    }
    if (st == WCT_OK) st = dev_alloc(s, (void **)&ps.phase_act, (size_t)(n_phases + 1) * ps.g.n_wires);
    if (st == WCT_OK) {
        const int tiles_w = (n_phases * ps.g.n_wires + ps.pp.tile_w - 1) / ps.pp.tile_w;
        ps.phase_tiles = tiles_w * ps.pp.n_tiles_t;
        ps.phase_flag_bytes = sizeof(uint32_t) * (2 * (size_t)ps.phase_tiles + 2);
        st = dev_alloc(s, (void **)&ps.phase_flags, ps.phase_flag_bytes);
    }
    if (st == WCT_OK && s->det) {
        ps.phase_grid64_bytes = 2 * ps.phase_grid_bytes;
        st = dev_alloc(s, (void **)&ps.phase_grids64, ps.phase_grid64_bytes);
        if (st == WCT_OK && cudaMemset(ps.phase_grids64, 0, ps.phase_grid64_bytes) != cudaSuccess)
            st = fail(s, WCT_ECUDA, "phase grid init");
    }
    if (st == WCT_OK) {
        cudaError_t e = cudaMemset(ps.phase_grids, 0, ps.phase_grid_bytes);
        if (e == cudaSuccess) e = cudaMemset(ps.phase_flags, 0, ps.phase_flag_bytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(s, e, "phase grid init");
    }
    const size_t need_imp = (size_t)n_phases * need;
    if (st == WCT_OK && need_imp > s->spec_imp_elems) {
        dev_free(s, s->spec_imp, sizeof(float2) * s->spec_imp_elems);
        s->spec_imp = nullptr;
        s->spec_imp_elems = 0;
        st = dev_alloc(s, (void **)&s->spec_imp, sizeof(float2) * need_imp);
        if (st == WCT_OK) s->spec_imp_elems = need_imp;
    }
    if (st) {
        drop_impact(s, ps);
        return st;
    }
    ps.n_phases = n_phases;
    return WCT_OK;
}

wct_status_t wct_sim_convolve_impact(wct_sim_t *s, int plane, const float *phase_grids, float *waveform, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    PlaneState &ps = s->planes[plane];
    if (ps.n_phases == 0) return fail(s, WCT_EINVAL, "plane has no impact responses");
    if (!phase_grids || !waveform) return fail(s, WCT_EINVAL, "phase_grids and waveform are required");
    cudaStream_t cs = (cudaStream_t)stream;
    const int nw = ps.g.n_wires, nt = ps.g.n_ticks;
    cudaError_t e = launch_row_r2c(ps.fft_imp, phase_grids, nt, nt, ps.n_phases * nw, s->spec_imp, cs, s->status);
    if (e == cudaSuccess)
        e = launch_wire_stage(ps.fft_imp, s->spec_imp, ps.resp_imp, nw, s->spec2, cs, s->status, nullptr, false,
                              ps.n_phases);
    if (e == cudaSuccess) e = launch_row_c2r(ps.fft_imp, s->spec2, nw, waveform, nt, nt, cs, s->status);
    if (e != cudaSuccess) return cuda_fail(s, e, "convolve impact");
    s->launches += 3;
    return WCT_OK;
}

wct_status_t wct_sim_digitize(wct_sim_t *s, int plane, const float *waveform, int16_t *adc, const wct_adc_t *params,
                              uint64_t event_id, void *stream) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    if (!waveform || !adc || !params) return fail(s, WCT_EINVAL, "waveform, adc and params are required");
    const wct_adc_t &a = *params;
    if (!std::isfinite(a.gain) || !std::isfinite(a.baseline) || !std::isfinite(a.noise_rms) || a.noise_rms < 0 ||
        a.bits < 1 || a.bits > 15)
        return fail(s, WCT_EINVAL, "bad digitiser parameters (finite gain / baseline, noise_rms >= 0, 1 <= bits <= 15)");
    const PlaneState &ps = s->planes[plane];
    AdcParams ap{};
    ap.gain = (float)a.gain;
    ap.baseline = (float)a.baseline;
    ap.noise_rms = (float)a.noise_rms;
    ap.max_code = (float)((1 << a.bits) - 1);
    ap.add_noise = a.add_noise && a.noise_rms > 0 ? 1 : 0;
    for (int k = 0; k < 20; ++k) ap.rk[k] = ps.pp.rk[k];
    ap.noise_wave = nullptr;
    const uint32_t c3 = ((uint32_t)(0x80 | plane) << 24) | ((uint32_t)event_id & 0xFFFFFFu);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (ap.add_noise && ps.noise_amp) {
        // coloured noise: spectrum from the plane's amplitudes, inverse row transform (the
        // transform's 1/M folded into the scale), then added by the digitiser
        FFTPlan full = ps.fft;
        full.Fs = full.Fu = (int32_t)((full.M + 2) & ~1);
        e = launch_noise_spectrum(ps.noise_amp, full.F, full.M, ps.g.n_wires, full.Fs, ap.noise_rms / (float)full.M, ap,
                                  c3, ps.noise_spec, cs);
        if (e == cudaSuccess)
            e = launch_row_c2r(full, ps.noise_spec, ps.g.n_wires, ps.noise_wave, ps.g.n_ticks, ps.g.n_ticks, cs, s->status);
        ap.noise_wave = ps.noise_wave;
        s->launches += 2;
    }
    if (e == cudaSuccess) e = launch_digitize(waveform, adc, ps.g.n_wires, ps.g.n_ticks, ap, c3, cs);
    if (e != cudaSuccess) return cuda_fail(s, e, "digitize");
    s->launches += 1;
    return WCT_OK;
}

wct_status_t wct_sim_set_noise_spectrum(wct_sim_t *s, int plane, const float *amplitude, int n_bins) {
    wct_status_t st = plane_check(s, plane);
    if (st) return st;
    PlaneState &ps = s->planes[plane];
    cudaDeviceSynchronize();                           // nothing may still use the old buffers
    dev_free(s, ps.noise_amp, ps.noise_bytes[0]);
    dev_free(s, ps.noise_spec, ps.noise_bytes[1]);
    dev_free(s, ps.noise_wave, ps.noise_bytes[2]);
    ps.noise_amp = nullptr;
    ps.noise_spec = nullptr;
    ps.noise_wave = nullptr;
    ps.noise_bytes[0] = ps.noise_bytes[1] = ps.noise_bytes[2] = 0;
    if (!amplitude) return WCT_OK;                     // back to white noise
    if (n_bins != ps.fft.F) return fail(s, WCT_EINVAL, "n_bins must equal the plane's spectrum bins (fft_length / 2 + 1)");
    for (int f = 0; f < n_bins; ++f)
        if (!std::isfinite(amplitude[f]) || amplitude[f] < 0.f) return fail(s, WCT_EINVAL, "amplitudes must be finite and >= 0");
    const size_t fs_full = (size_t)((ps.fft.M + 2) & ~1);
    const size_t bytes[3] = {sizeof(float) * (size_t)n_bins, sizeof(float2) * (size_t)ps.g.n_wires * fs_full,
                             sizeof(float) * (size_t)ps.g.n_wires * ps.g.n_ticks};
    void **ptr[3] = {(void **)&ps.noise_amp, (void **)&ps.noise_spec, (void **)&ps.noise_wave};
    for (int k = 0; k < 3 && st == WCT_OK; ++k) {
        st = dev_alloc(s, ptr[k], bytes[k]);
        if (st == WCT_OK) ps.noise_bytes[k] = bytes[k];
    }
    if (st == WCT_OK) {
        const cudaError_t e = cudaMemcpy(ps.noise_amp, amplitude, bytes[0], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(s, e, "noise spectrum");
    }
    if (st) {
        dev_free(s, ps.noise_amp, ps.noise_bytes[0]);
        dev_free(s, ps.noise_spec, ps.noise_bytes[1]);
        dev_free(s, ps.noise_wave, ps.noise_bytes[2]);
        ps.noise_amp = nullptr;
        ps.noise_spec = nullptr;
        ps.noise_wave = nullptr;
        ps.noise_bytes[0] = ps.noise_bytes[1] = ps.noise_bytes[2] = 0;
    }
    return st;
}

wct_status_t wct_sim_set_lifetime(wct_sim_t *s, double lifetime_us, int32_t fluctuate) {
    if (!s) return WCT_EINVAL;
    if (std::isnan(lifetime_us)) return fail(s, WCT_EINVAL, "lifetime is NaN");
    const bool on = lifetime_us > 0.0 && std::isfinite(lifetime_us);
    cudaDeviceSynchronize();                           // launches in flight keep the old value
    for (int p = 0; p < s->n_planes; ++p) {
        PlaneParams &pp = s->planes[p].pp;
        pp.inv_v_lifetime = on ? (float)(1.0 / (pp.v * lifetime_us)) : 0.f;
        pp.fluct_absorb = on && fluctuate ? 1 : 0;
    }
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);   // recorded batches captured the old value
    s->graphs.clear();
    s->seen.clear();
    return WCT_OK;
}

wct_status_t wct_sim_sync(wct_sim_t *s, void *stream) {
    if (!s) return WCT_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream sync");
    int32_t code = 0;
    e = cudaMemcpy(&code, s->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(int32_t));
    if (e == cudaSuccess && code != 0) {
        // a device-side error may have left a grid tile uncleared: restore the all-zero grids
        clear_grids(s);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "status read");
    if (code == ST_EINVAL) return fail(s, WCT_EINVAL, "invalid depo(s) skipped (non-finite, x<0, q<0 or window too large)");
    if (code == ST_ETIMEOUT) return fail(s, WCT_ETIMEOUT, "a device-side wait timed out");
    if (code != 0) return fail(s, WCT_EDEVICE, "device-side error");
    return WCT_OK;
}

wct_status_t wct_sim_plane_info(const wct_sim_t *s, int plane, int64_t *info) {
    if (!s || !info || plane < 0 || plane >= s->n_planes) return WCT_EINVAL;
    const PlaneState &ps = s->planes[plane];
    info[0] = ps.g.n_wires;
    info[1] = ps.g.n_ticks;
    info[2] = ps.fft.fft_len;
    info[3] = ps.fft.F;
    info[4] = ps.fft.Fs;
    info[5] = ps.pp.tile_w;
    info[6] = ps.pp.tile_t;
    info[7] = ps.n_tiles;
    info[8] = ps.fft.Fu;
    return WCT_OK;
}

wct_status_t wct_sim_set_timing(wct_sim_t *s, int enable) {
    if (!s) return WCT_EINVAL;
    s->timing = enable != 0;
    s->slots_used = 0;
    s->events_timed = 0;
    s->bslots_used = 0;
    s->batches_timed = 0;
    return WCT_OK;
}

wct_status_t wct_sim_stage_times(wct_sim_t *s, float *us, int n) {
    if (!s || !us || n < 0) return WCT_EINVAL;
    double acc[kStages] = {0, 0, 0, 0, 0};
    for (int k = 0; k < s->slots_used; ++k) {
        auto &ev = s->slots[k];
        cudaError_t e = cudaEventSynchronize(ev[kStages]);
        if (e != cudaSuccess) return cuda_fail(s, e, "stage events");
        for (int j = 0; j < kStages; ++j) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[j], ev[j + 1]) == cudaSuccess) acc[j] += 1000.0 * ms;
            else cudaGetLastError();
        }
    }
    const double div = s->events_timed > 0 ? (double)s->events_timed : 1.0;
    for (int j = 0; j < n && j < kStages; ++j) us[j] = (float)(acc[j] / div);
    if (n > kStages) us[kStages] = (float)s->events_timed;
    if (n > kStages + 3) {
        double raster = 0.0, conv = 0.0;
        auto span = [](cudaEvent_t a, cudaEvent_t b) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                cudaGetLastError();
                return 0.0;
            }
            return 1000.0 * ms;
        };
        for (int k = 0; k < s->bslots_used; ++k) {
            auto &ev = s->bslots[k];
            for (int j : {1, 3, 5}) {
                cudaError_t e = cudaEventSynchronize(ev[j]);
                if (e != cudaSuccess) return cuda_fail(s, e, "batch stage events");
            }
            raster += span(ev[0], ev[1]);
            conv += std::max(span(ev[2], ev[3]), span(ev[4], ev[5]));
        }
        const double bdiv = s->batches_timed > 0 ? (double)s->batches_timed : 1.0;
        us[kStages + 1] = (float)(raster / bdiv);
        us[kStages + 2] = (float)(conv / bdiv);
        us[kStages + 3] = (float)s->batches_timed;
    }
    return WCT_OK;
}

wct_status_t wct_sim_counters(const wct_sim_t *s, int64_t *out, int n) {
    if (!s || !out || n < 0) return WCT_EINVAL;
    if (n > 0) out[0] = s->launches;
    if (n > 1) out[1] = (int64_t)s->bytes;
    if (n > 2) out[2] = s->graph_launches;
    return WCT_OK;
}

const char *wct_sim_last_error(const wct_sim_t *s) { return s ? s->err.c_str() : "null handle"; }

wct_status_t wct_sim_selftest_wait(wct_sim_t *s, int64_t limit_cycles, void *stream) {
    if (!s || limit_cycles < 0) return WCT_EINVAL;
    cudaError_t e = launch_wait_selftest((long long)limit_cycles, s->status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "wait self-test");
    return WCT_OK;
}

wct_status_t wct_debug_bounds(wct_sim_t *s, int64_t *out) {
    if (!s || !out) return WCT_EINVAL;
    int32_t rec[3] = {0, 0, 0};
    const cudaError_t e = cudaMemcpy(rec, s->status + 1, sizeof(rec), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "bounds record");
    for (int k = 0; k < 3; ++k) out[k] = rec[k];
#ifdef WCT_BOUNDS_CHECK
    return WCT_OK;
#else
    return WCT_EINVAL;   // not a bounds-checked build: nothing is recorded
#endif
}

wct_status_t wct_debug_fail_alloc(int64_t n) {
    g_fail_alloc.store(n < 0 ? -1 : (long long)n);
    return WCT_OK;
}

wct_status_t wct_philox4x32_10(const uint32_t *ctr, uint64_t seed, int64_t n, uint32_t *out, void *stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return WCT_EINVAL;
    if (((uintptr_t)ctr & 15) || ((uintptr_t)out & 15)) return WCT_EINVAL;
    cudaError_t e = launch_philox(ctr, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), n, out,
                                  (cudaStream_t)stream);
    return e == cudaSuccess ? WCT_OK : WCT_ECUDA;
}

// ------------------------------------------------------------------------------------------
// Convolution that allocates nothing: its scratch is a fixed array reserved in device memory
// when the library is loaded.  For callers that may not allocate device memory at call time.
// ------------------------------------------------------------------------------------------
}  // extern "C"

namespace {

constexpr size_t kStaticElems = (size_t)WCT_CONVOLVE_STATIC_SCRATCH_BYTES / sizeof(float2);
constexpr size_t kStaticHead = 32;   // float2 = 256 bytes at the head: the status word (+ bounds record)
constexpr int kMaxDevices = 64;
__device__ __align__(256) float2 g_convolve_scratch[kStaticElems];

std::mutex g_static_mu;
float2 *g_static_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Looked up once per device
// (with that device current) and cached, and the status word at its head cleared then; the
// name g_convolve_scratch itself is only a host-side stand-in and must never be passed to a
// kernel.
cudaError_t static_scratch(float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_convolve_scratch);
        if (e != cudaSuccess) return e;
        e = cudaMemset(p, 0, sizeof(float2) * kStaticHead);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = static_cast<float2 *>(p);
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

size_t round_up_256(size_t n_float2) { return (n_float2 + 31) & ~(size_t)31; }   // 32 float2 = 256 B

}  // namespace

extern "C" {

wct_status_t wct_convolve_static(const float *grid, int32_t n_wires, int32_t n_ticks, const float *response,
                                 int32_t n_wires_resp, int32_t n_ticks_resp, float *waveform, void *stream) {
    if (!grid || !response || !waveform) return WCT_EINVAL;
    if (n_wires < 1 || n_ticks < 1 || n_wires_resp < 1 || (n_wires_resp & 1) == 0 ||
        n_wires_resp > WCT_MAX_RESPONSE_WIRES || n_ticks_resp < 1 || n_ticks_resp > 65536)
        return WCT_EINVAL;
    FFTPlan p{};
    if (!plan_fft(n_ticks, n_ticks_resp, p)) return WCT_EINVAL;
    const int KW = WCT_MAX_RESPONSE_WIRES;
    const size_t n_tw = round_up_256((size_t)p.M), n_rtw = round_up_256((size_t)p.M + 1);
    const size_t n_resp = round_up_256((size_t)KW * p.Fs);
    const size_t n_spec = round_up_256((size_t)n_wires * p.Fs);
    if (kStaticHead + n_tw + n_rtw + n_resp + 2 * n_spec > kStaticElems) return WCT_EINVAL;   // beyond the scratch
    float2 *base = nullptr;
    if (static_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return WCT_ECUDA;
    }
    // the kernels' bounded waits record a timeout here (it stays set until read by
    // wct_convolve_static_status)
    int32_t *status = reinterpret_cast<int32_t *>(base);
    p.tw = base + kStaticHead;
    p.rtw = p.tw + n_tw;
    float2 *resp_spec = p.rtw + n_rtw;
    float2 *S = resp_spec + n_resp;
    float2 *T = S + n_spec;
    cudaStream_t cs = (cudaStream_t)stream;
    const int off = (KW - n_wires_resp) / 2;
    cudaError_t e = launch_make_twiddles(p, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(resp_spec, 0, sizeof(float2) * (size_t)KW * p.Fs, cs);
    if (e == cudaSuccess)
        e = launch_row_r2c(p, response, n_ticks_resp, n_ticks_resp, n_wires_resp, resp_spec + (size_t)off * p.Fs, cs,
                           status);
    if (e == cudaSuccess) e = launch_scale_spectrum(resp_spec, (int64_t)KW * p.Fs, 1.0f / (float)p.M, cs);
    if (e == cudaSuccess) e = launch_row_r2c(p, grid, n_ticks, n_ticks, n_wires, S, cs, status);
    if (e == cudaSuccess) e = launch_wire_stage(p, S, resp_spec, n_wires, T, cs, status);
    if (e == cudaSuccess) e = launch_row_c2r(p, T, n_wires, waveform, n_ticks, n_ticks, cs, status);
    return e == cudaSuccess ? WCT_OK : WCT_ECUDA;
}

wct_status_t wct_convolve_static_status(void *stream) {
    float2 *base = nullptr;
    if (static_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return WCT_ECUDA;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int32_t code = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&code, base, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && code != 0) e = cudaMemset(base, 0, sizeof(float2) * kStaticHead);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return WCT_ECUDA;
    }
    if (code == ST_ETIMEOUT) return WCT_ETIMEOUT;
    return code == 0 ? WCT_OK : WCT_EDEVICE;
}

wct_status_t wct_convolve_static_selftest_wait(int64_t limit_cycles, void *stream) {
    if (limit_cycles < 0) return WCT_EINVAL;
    float2 *base = nullptr;
    if (static_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return WCT_ECUDA;
    }
    const cudaError_t e =
        launch_wait_selftest((long long)limit_cycles, reinterpret_cast<int32_t *>(base), (cudaStream_t)stream);
    return e == cudaSuccess ? WCT_OK : WCT_ECUDA;
}

}  // extern "C"
