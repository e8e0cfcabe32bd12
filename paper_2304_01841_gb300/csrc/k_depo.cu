// Depo preparation (drift, diffusion, +-n sigma windows), tile binning and prefix scans.
//
// The paper (§2) bins "individual ionization electron groups" into patches after they
// drift to the wires; the Kokkos port computes the patch offsets with a device prefix
// scan, which the OpenMP port removed (§4.3).  Here:
//   k_prep      one thread per depo: FP64 drift / diffusion, window bounds, a 32-byte
//               descriptor, and a count of the output tiles the window overlaps;
//   k_bin_patches / k_fill_patches  tile binning of caller-supplied patch descriptors;
//   scans       three-phase exclusive scans (tile-list offsets, patch offsets).
#include "wct_internal.cuh"
#include "wct_device.cuh"

namespace wct {

namespace {

constexpr int kPrepThreads = 256;

struct TileRange {
    int tw0, tw1, tt0, tt1;   // inclusive; tw0 > tw1 when empty
};

__device__ __forceinline__ TileRange tile_range(int lo_t, int nt, int lo_p, int np, const PlaneParams &pp) {
    TileRange r{0, -1, 0, -1};
    if (nt <= 0 || np <= 0) return r;
    int w0 = floor_div(lo_p, pp.n_imp);
    int w1 = floor_div(lo_p + np - 1, pp.n_imp);
    int t0 = lo_t, t1 = lo_t + nt - 1;
    w0 = max(w0, 0);
    w1 = min(w1, pp.n_wires - 1);
    t0 = max(t0, 0);
    t1 = min(t1, pp.n_ticks - 1);
    if (w0 > w1 || t0 > t1) return r;
    r.tw0 = w0 / pp.tile_w;
    r.tw1 = w1 / pp.tile_w;
    r.tt0 = t0 / pp.tile_t;
    r.tt1 = t1 / pp.tile_t;
    return r;
}

__global__ void __launch_bounds__(kPrepThreads)
k_prep(const float *__restrict__ t0, const float *__restrict__ x, const float *__restrict__ y,
       const float *__restrict__ z, const float *__restrict__ q, int64_t n, PlaneParams pp,
       DepoDesc *__restrict__ desc, int32_t *__restrict__ tile_count, int64_t *__restrict__ patch_size,
       int32_t *status, uint32_t event_lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DepoDesc d;
    const bool ok = depo_window(t0[i], x[i], y[i], z[i], q[i], pp, d);
    if (!ok) set_status(status, ST_EINVAL);
    else d.q = drift_absorb(d.q, x[i], (uint32_t)i, event_lo, pp);
    desc[i] = d;
    if (patch_size) patch_size[i] = (int64_t)d.nt * (int64_t)d.np;
    if (tile_count) {
        const TileRange r = tile_range(d.lo_t, d.nt, d.lo_p, d.np, pp);
        for (int tw = r.tw0; tw <= r.tw1; ++tw)
            for (int tt = r.tt0; tt <= r.tt1; ++tt) atomicAdd(&tile_count[tw * pp.n_tiles_t + tt], 1);
    }
}

// A caller-supplied patch descriptor is usable if its window is within the library limits.
__device__ __forceinline__ bool pd_ok(const int64_t *e) {
    return e[3] >= 0 && e[3] <= WCT_MAX_WINDOW_TICKS && e[4] >= 0 && e[4] <= WCT_MAX_WINDOW_IMPACTS &&
           e[1] >= -(1LL << 30) && e[1] <= (1LL << 30) && e[2] >= -(1LL << 30) && e[2] <= (1LL << 30);
}

// Tile binning from caller-supplied patch descriptors {offset, lo_t, lo_p, nt, np}.
__global__ void __launch_bounds__(kPrepThreads)
k_bin_patches(int64_t n, const int64_t *__restrict__ pd, PlaneParams pp, int32_t *__restrict__ tile_count,
              int32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t *e = pd + 5 * i;
    if (!pd_ok(e)) {
        set_status(status, ST_EINVAL);
        return;
    }
    const TileRange r = tile_range((int)e[1], (int)e[3], (int)e[2], (int)e[4], pp);
    for (int tw = r.tw0; tw <= r.tw1; ++tw)
        for (int tt = r.tt0; tt <= r.tt1; ++tt) atomicAdd(&tile_count[tw * pp.n_tiles_t + tt], 1);
}

__global__ void __launch_bounds__(kPrepThreads)
k_fill_patches(int64_t n, const int64_t *__restrict__ pd, PlaneParams pp, const int32_t *__restrict__ tile_off,
               int32_t *__restrict__ cursor, int32_t *__restrict__ list, int64_t list_cap, int32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t *e = pd + 5 * i;
    if (!pd_ok(e)) return;
    const TileRange r = tile_range((int)e[1], (int)e[3], (int)e[2], (int)e[4], pp);
    for (int tw = r.tw0; tw <= r.tw1; ++tw)
        for (int tt = r.tt0; tt <= r.tt1; ++tt) {
            const int tile = tw * pp.n_tiles_t + tt;
            const int64_t pos = (int64_t)tile_off[tile] + atomicAdd(&cursor[tile], 1);
            if (pos < list_cap) list[pos] = (int32_t)i;
            else set_status(status, ST_EDEVICE);
        }
}

// ---- exclusive scan: out[0..n] with out[n] = total --------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T &total) {
    __shared__ T warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    T wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const T t = warp_tot[w];
        if (w < warp) wbase += t;
        tot += t;
    }
    __syncthreads();
    total = tot;
    return wbase + inc - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_block(const T *__restrict__ in, T *__restrict__ out, int64_t n, T *__restrict__ block_sums) {
    __shared__ T buf[kScanBlock];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads) {
        const int64_t idx = base + k;
        buf[k] = idx < n ? in[idx] : T(0);
    }
    __syncthreads();
    T v[kScanItems];
    T run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = run;
        run += buf[threadIdx.x * kScanItems + k];
    }
    T total;
    const T pre = block_exclusive<T>(run, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) buf[threadIdx.x * kScanItems + k] = pre + v[k];
    __syncthreads();
    for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads) {
        const int64_t idx = base + k;
        if (idx < n) out[idx] = buf[k];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums in chunks, with a running carry.
template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(T *__restrict__ sums, int64_t nb, T *__restrict__ out, int64_t n) {
    T carry = 0;
    for (int64_t c = 0; c < nb; c += kScanThreads) {
        const int64_t idx = c + threadIdx.x;
        const T v = idx < nb ? sums[idx] : T(0);
        T total;
        const T pre = block_exclusive<T>(v, total);
        if (idx < nb) sums[idx] = carry + pre;
        carry += total;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_add(T *__restrict__ out, int64_t n, const T *__restrict__ sums) {
    const T add = sums[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads) {
        const int64_t idx = base + k;
        if (idx < n) out[idx] += add;
    }
}

template <typename T>
cudaError_t scan_impl(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) {
        k_scan_sums<T><<<1, kScanThreads, 0, s>>>(tmp, 0, out, 0);
        return cudaGetLastError();
    }
    k_scan_block<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    k_scan_sums<T><<<1, kScanThreads, 0, s>>>(tmp, nb, out, n);
    k_scan_add<T><<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, tmp);
    return cudaGetLastError();
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, tmp, s);
}
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, tmp, s);
}

cudaError_t launch_prep(const wct_depos_t &d, const PlaneParams &pp, DepoDesc *desc, int32_t *tile_count,
                        int64_t *patch_size, int32_t *status, cudaStream_t s) {
    if (d.n <= 0) return cudaSuccess;
    k_prep<<<blocks_for(d.n, kPrepThreads), kPrepThreads, 0, s>>>(d.t0_us, d.x_mm, d.y_mm, d.z_mm, d.q_e, d.n, pp,
                                                                   desc, tile_count, patch_size, status,
                                                                   (uint32_t)d.event_id);
    return cudaGetLastError();
}

cudaError_t launch_bin_patches(int64_t n, const int64_t *patch_desc, const PlaneParams &pp, int32_t *tile_count,
                               int32_t *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bin_patches<<<blocks_for(n, kPrepThreads), kPrepThreads, 0, s>>>(n, patch_desc, pp, tile_count, status);
    return cudaGetLastError();
}

cudaError_t launch_fill_patches(int64_t n, const int64_t *patch_desc, const PlaneParams &pp, const int32_t *tile_off,
                                int32_t *tile_cursor, int32_t *tile_list, int64_t list_cap, int32_t *status,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill_patches<<<blocks_for(n, kPrepThreads), kPrepThreads, 0, s>>>(n, patch_desc, pp, tile_off, tile_cursor,
                                                                         tile_list, list_cap, status);
    return cudaGetLastError();
}

}  // namespace wct
