// Device-side helpers: Philox4x32-10, Box-Muller, integer floor division, status flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "wct_internal.cuh"

namespace wct {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each of the ten rounds multiplies
// counter words 0 and 2 by the round multipliers, keeps the high and low halves, and mixes
// them with words 1 and 3 and the key; the key advances by the Weyl increments between
// rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator with the ten round keys precomputed (rk[2r], rk[2r+1] = key + r * Weyl),
// so each round's key is an operand instead of two additions.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per word gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                       (uint32_t)p0);
    }
    return c;
}

// Two standard normals from two 32-bit words (Box-Muller): u = (x + 1/2) 2^-32 in (0,1),
// r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b).  Evaluated with the SFU's
// approximate lg2 / sqrt / sin / cos instructions (relative errors ~2^-22, absolute sin/cos
// error ~2^-20.5 on [-pi, pi]); the angle is reduced to (-pi, pi) first, using
// cos(t) = -cos(t - pi) and sin(t) = -sin(t - pi).  The resulting deviates differ from an
// FP64 evaluation by < 1e-5 absolute, far inside the patch / grid tolerance.
__device__ __forceinline__ float sfu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_sin(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_cos(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float s32 = 2.3283064365386963e-10f;   // 2^-32
    const float h32 = 1.1641532182693481e-10f;   // 2^-33
    const float ua = fmaf(__uint2float_rn(a), s32, h32);
    const float ub = fmaf(__uint2float_rn(b), s32, h32);
    const float m2ln2 = -1.3862943611198906f;    // -2 ln 2
    const float r = sfu_sqrt(fmaxf(m2ln2 * sfu_lg2(ua), 0.f));
    const float t = 6.283185307179586f * (ub - 0.5f);   // 2 pi u_b - pi, in (-pi, pi)
    return make_float2(-r * sfu_cos(t), -r * sfu_sin(t));
}

// Drift attenuation by the electron lifetime (the step before rasterization): the surviving
// charge is Binomial(q, p) with p = exp(-t_d / lifetime), t_d = x / v; without fluctuation its
// mean q p, with fluctuation its normal approximation max(0, q p + sqrt(q p (1 - p)) z), z the
// first Box-Muller normal of Philox(depo, 0, 0, 0xFF << 24 | event) under the seed's key (plane
// field 0xFF: no bin of any plane uses it, and every plane sees the same surviving charge).
__device__ __forceinline__ float drift_absorb(float q, float x, uint32_t depo, uint32_t event_lo,
                                              const PlaneParams &pp) {
    if (pp.inv_v_lifetime == 0.f) return q;
    const float p = expf(-x * pp.inv_v_lifetime);
    const float m = q * p;
    if (!pp.fluct_absorb) return m;
    const uint4 w = philox4x32_10_rk(make_uint4(depo, 0u, 0u, (0xFFu << 24) | (event_lo & 0xFFFFFFu)), pp.rk);
    const float z = box_muller(w.x, w.y).x;
    return fmaxf(fmaf(sqrtf(m * (1.f - p)), z, m), 0.f);
}

__device__ __forceinline__ int floor_div(int a, int b) {   // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

// Bounds-checked build (-DWCT_BOUNDS_CHECK, a debugging aid in place of a memory checker): the
// computed indices of the scatter targets, shared-memory boxes, ring slots, tile clears and
// conversions are checked before use.  A violation skips the access, sets the status word to
// WCT_EDEVICE and records the first (source line, index, limit) in status[1..3] (read by
// wct_debug_bounds).  The release build compiles every check to `true`.
#ifdef WCT_BOUNDS_CHECK
static __device__ __noinline__ bool bounds_fail(int32_t *status, long long i, long long n, int line) {
    if (status) {
        atomicCAS(status, 0, ST_EDEVICE);
        if (atomicCAS(status + 1, 0, line) == 0) {
            status[2] = (int32_t)i;
            status[3] = (int32_t)n;
        }
    }
    return false;
}
#define WCT_IDX_OK(status, i, n) \
    ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ? true \
                                                                             : bounds_fail((status), (i), (n), __LINE__))
#else
#define WCT_IDX_OK(status, i, n) true
#endif

// +-nsigma window on one axis, decided in FP64 with explicitly rounded operations so the
// bounds match a host FP64 evaluation of the same expressions bit for bit.
__device__ __forceinline__ void axis_window(double mu, double s, double nsigma, long long &lo, long long &n) {
    if (s < 1e-6) {
        lo = (long long)floor(mu);
        n = 1;
        return;
    }
    const double ns = __dmul_rn(nsigma, s);
    const double a = __dsub_rn(mu, ns);
    const double b = __dadd_rn(mu, ns);
    lo = (long long)floor(a);
    n = (long long)floor(b) - lo + 1;
}

// Drift, diffusion and +-nsigma window of one depo (FP64), packed into a DepoDesc.
// Returns false (and an empty descriptor) for an invalid depo: a non-finite value, x < 0,
// q < 0, a window over the limits, or one that starts more than 2^30 bins from the origin.
//   t_d = x / v, arrival = t0 + t_d, sigma_L,T = sqrt(2 D_L,T t_d)
//   mu_t = (arrival - t_window0) / tick, s_t = (sigma_L / v) / tick
//   mu_p = (z cos a + y sin a - origin) / (pitch / n_imp), s_p = sigma_T / (pitch / n_imp)
__device__ __forceinline__ bool depo_window_f64(double T0, double X, double Y, double Z, double Q,
                                                const PlaneParams &pp, DepoDesc &d) {
    d.mu_t = d.mu_p = d.inv_t = d.inv_p = 0.f;
    d.q = 0.f;
    d.lo_t = d.lo_p = 0;
    d.nt = d.np = 0;
    bool ok = isfinite(T0) && isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(Q) && X >= 0.0 && Q >= 0.0;
    if (!ok) return false;
    const double td = __ddiv_rn(X, pp.v);
    const double arrival = __dadd_rn(T0, td);
    const double sigL = __dsqrt_rn(__dmul_rn(__dmul_rn(2.0, pp.DL), td));
    const double sigT = __dsqrt_rn(__dmul_rn(__dmul_rn(2.0, pp.DT), td));
    const double mu_t = __ddiv_rn(__dsub_rn(arrival, pp.tw0), pp.tick);
    const double s_t = __ddiv_rn(__ddiv_rn(sigL, pp.v), pp.tick);
    const double p = __dadd_rn(__dmul_rn(Z, pp.cos_a), __dmul_rn(Y, pp.sin_a));
    const double mu_p = __ddiv_rn(__dsub_rn(p, pp.origin), pp.dp);
    const double s_p = __ddiv_rn(sigT, pp.dp);
    const double big = 1099511627776.0;   // 2^40 bins: keeps floor() within int64
    if (!(fabs(mu_t) < big && fabs(mu_p) < big && s_t < big && s_p < big)) return false;
    long long lo_t = 0, n_t = 0, lo_p = 0, n_p = 0;
    axis_window(mu_t, s_t, pp.nsigma, lo_t, n_t);
    axis_window(mu_p, s_p, pp.nsigma, lo_p, n_p);
    const long long lim = 1LL << 30;
    if (n_t > WCT_MAX_WINDOW_TICKS || n_p > WCT_MAX_WINDOW_IMPACTS || lo_t < -lim || lo_t > lim || lo_p < -lim ||
        lo_p > lim)
        return false;
    d.lo_t = (int32_t)lo_t;
    d.lo_p = (int32_t)lo_p;
    d.nt = (int16_t)n_t;
    d.np = (int16_t)n_p;
    d.mu_t = (float)__dsub_rn(mu_t, (double)lo_t);
    d.mu_p = (float)__dsub_rn(mu_p, (double)lo_p);
    d.inv_t = (s_t < 1e-6) ? 0.f : (float)__drcp_rn(__dmul_rn(1.4142135623730951, s_t));
    d.inv_p = (s_p < 1e-6) ? 0.f : (float)__drcp_rn(__dmul_rn(1.4142135623730951, s_p));
    d.q = (float)Q;
    return true;
}

// Packed FP32 pair arithmetic (sm_100+ f32x2): one instruction for both lanes of a float2.
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {   // a * b + c, lane-wise
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return bits_f2(d);
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}

// Double-float arithmetic (an unevaluated sum hi + lo of two floats, ~48-bit significand)
// from error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based
// TwoProduct.  Explicitly rounded operations keep the compiler from contracting them.
struct ffloat {
    float hi, lo;
};
__device__ __forceinline__ ffloat ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ffloat ff_fast_two_sum(float a, float b) {   // |a| >= |b| (or a == 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ffloat ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
    ffloat s = ff_two_sum(a.hi, b.hi);
    const ffloat t = ff_two_sum(a.lo, b.lo);
    s = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ ffloat ff_mul(ffloat a, ffloat b) {
    ffloat p = ff_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ffloat ff_mul_f(float a, ffloat b) {
    ffloat p = ff_two_prod(a, b.hi);
    p.lo = __fmaf_rn(a, b.lo, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ffloat ff_of(const float (&c)[2]) { return {c[0], c[1]}; }
__device__ __forceinline__ ffloat ff_neg(ffloat a) { return {-a.hi, -a.lo}; }

// floor(v) when v = hi + lo lies more than eps from every integer (|hi| < 2^22); false
// otherwise.  hi - floor(hi) and floor(hi) + 1 - hi are exact.
__device__ __forceinline__ bool ff_floor(ffloat v, float eps, int &f) {
    if (!(fabsf(v.hi) < 4194304.f)) return false;
    const float fl = floorf(v.hi);
    const float above = __fadd_rn(__fsub_rn(v.hi, fl), v.lo);
    const float below = __fsub_rn(__fsub_rn(__fadd_rn(fl, 1.f), v.hi), v.lo);
    f = (int)fl;
    return above > eps && below > eps;
}

// The same window, decided cheaply.  FP64 arithmetic is slow on this part, so the fast
// path is all FP32: mu_t = x / (v tick) + (t0 - tw0) / tick and mu_p = (z cos a + y sin a -
// origin) / dp in double-float arithmetic with host-computed reciprocals (error ~1e-13 of
// the operands' magnitude, against ~1e-16 for the FP64 evaluation), sigma from an FP32
// square root (relative error < 2^-21).  Each window edge floor(mu -+ n sigma) is accepted
// when it lies farther than eps from every integer, eps = 1e-9 (1 + the magnitudes summed) +
// 4e-6 n sigma bounding both evaluations' errors generously, and the point-charge test when
// sigma is not within 1e-5 (relative) of its threshold; otherwise depo_window_f64 decides,
// exactly as the oracle.  mu_t / mu_p relative to the window and the erf scales only feed
// FP32 weights.
__device__ __forceinline__ bool depo_window(float T0, float X, float Y, float Z, float Q, const PlaneParams &pp,
                                            DepoDesc &d) {
    const bool ok = isfinite(T0) && isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(Q) && X >= 0.f && Q >= 0.f;
    if (!ok) return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    // mu_t = X * inv_vtick + (T0 - tw0) * inv_tick
    const ffloat dt0 = ff_add({T0, 0.f}, ff_neg(ff_of(pp.ff[2])));
    const ffloat mu_t = ff_add(ff_mul_f(X, ff_of(pp.ff[0])), ff_mul(dt0, ff_of(pp.ff[1])));
    // mu_p = (Z cos a + Y sin a - origin) * inv_dp
    const ffloat pz = ff_add(ff_mul_f(Z, ff_of(pp.ff[3])), ff_mul_f(Y, ff_of(pp.ff[4])));
    const ffloat mu_p = ff_mul(ff_add(pz, ff_neg(ff_of(pp.ff[5]))), ff_of(pp.ff[6]));
    const float sx = sqrtf(X);
    const float s_t = sx * pp.kt, s_p = sx * pp.kp;
    const float ns = (float)pp.nsigma;
    if (!(s_t < 1e30f && s_p < 1e30f)) return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    const float mag_t = fabsf(mu_t.hi) + (fabsf(T0) + fabsf(pp.ff[2][0])) * pp.ff[1][0] + X * pp.ff[0][0];
    const float mag_p = fabsf(mu_p.hi) + (fabsf(pz.hi) + fabsf(pp.ff[5][0])) * pp.ff[6][0];
    const float et = 1e-9f * (1.f + mag_t) + 4e-6f * (ns * s_t);
    const float ep = 1e-9f * (1.f + mag_p) + 4e-6f * (ns * s_p);
    int lo_t, hi_t, lo_p, hi_p;
    bool sure = true;
    // point-charge threshold: sigma < 1e-6 bin
    const bool dt = s_t < 1e-6f, dp = s_p < 1e-6f;
    sure &= fabsf(s_t - 1e-6f) > 1e-11f && fabsf(s_p - 1e-6f) > 1e-11f;
    if (dt) sure &= ff_floor(mu_t, et, lo_t), hi_t = lo_t;
    else {
        sure &= ff_floor(ff_add(mu_t, {-(ns * s_t), 0.f}), et, lo_t);
        sure &= ff_floor(ff_add(mu_t, {ns * s_t, 0.f}), et, hi_t);
    }
    if (dp) sure &= ff_floor(mu_p, ep, lo_p), hi_p = lo_p;
    else {
        sure &= ff_floor(ff_add(mu_p, {-(ns * s_p), 0.f}), ep, lo_p);
        sure &= ff_floor(ff_add(mu_p, {ns * s_p, 0.f}), ep, hi_p);
    }
    if (!sure) return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    const int n_t = hi_t - lo_t + 1, n_p = hi_p - lo_p + 1;
    d.mu_t = d.mu_p = d.inv_t = d.inv_p = 0.f;
    d.q = 0.f;
    d.lo_t = d.lo_p = 0;
    d.nt = d.np = 0;
    if (n_t > WCT_MAX_WINDOW_TICKS || n_p > WCT_MAX_WINDOW_IMPACTS) return false;   // |edges| < 2^22 < 2^30
    d.lo_t = lo_t;
    d.lo_p = lo_p;
    d.nt = (int16_t)n_t;
    d.np = (int16_t)n_p;
    d.mu_t = __fadd_rn(__fsub_rn(mu_t.hi, (float)lo_t), mu_t.lo);
    d.mu_p = __fadd_rn(__fsub_rn(mu_p.hi, (float)lo_p), mu_p.lo);
    d.inv_t = dt ? 0.f : 0.70710678118654752f / s_t;
    d.inv_p = dp ? 0.f : 0.70710678118654752f / s_p;
    d.q = Q;
    return true;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace wct
