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
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
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

__device__ __forceinline__ int floor_div(int a, int b) {   // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

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

// The same window, decided cheaply.  FP64 division and square root are slow on this part,
// so: mu comes from multiplications by host-computed FP64 reciprocals (within ~1e-12 bin of
// the divided value), sigma from an FP32 square root (relative error < 2^-21).  Each window
// edge floor(mu -+ n sigma) is accepted when the interval of +-eps around it (eps bounds both
// errors generously) holds no integer, and the point-charge test when sigma is not within
// 1e-5 (relative) of its threshold; otherwise depo_window_f64 decides, exactly as before.
// mu_t/mu_p relative to the window and the erf scales only feed FP32 weights.
__device__ __forceinline__ bool fast_edge(double a, double eps, long long &f) {
    const double lo = floor(a - eps), hi = floor(a + eps);
    f = (long long)lo;
    return lo == hi;
}

__device__ __forceinline__ bool depo_window(double T0, double X, double Y, double Z, double Q, const PlaneParams &pp,
                                            DepoDesc &d) {
    const bool ok = isfinite(T0) && isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(Q) && X >= 0.0 && Q >= 0.0;
    if (!ok) return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    const double mu_t = fma(X, pp.inv_vtick, (T0 - pp.tw0) * pp.inv_tick);
    const double p = fma(Z, pp.cos_a, Y * pp.sin_a);
    const double mu_p = (p - pp.origin) * pp.inv_dp;
    const float sx = sqrtf((float)X);
    const float s_t = sx * pp.kt, s_p = sx * pp.kp;
    const float ns = (float)pp.nsigma;
    const double big = 1099511627776.0;
    if (!(fabs(mu_t) < 0.5 * big && fabs(mu_p) < 0.5 * big && s_t < 1e30f && s_p < 1e30f))
        return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    long long lo_t, hi_t, lo_p, hi_p;
    bool sure = true;
    // point-charge threshold: sigma < 1e-6 bin
    const bool dt = s_t < 1e-6f, dp = s_p < 1e-6f;
    sure &= fabsf(s_t - 1e-6f) > 1e-11f && fabsf(s_p - 1e-6f) > 1e-11f;
    const double et = 1e-9 * (1.0 + fabs(mu_t)) + 4e-6 * (double)(ns * s_t);
    const double ep = 1e-9 * (1.0 + fabs(mu_p)) + 4e-6 * (double)(ns * s_p);
    if (dt) sure &= fast_edge(mu_t, et, lo_t), hi_t = lo_t;
    else {
        sure &= fast_edge(mu_t - (double)(ns * s_t), et, lo_t);
        sure &= fast_edge(mu_t + (double)(ns * s_t), et, hi_t);
    }
    if (dp) sure &= fast_edge(mu_p, ep, lo_p), hi_p = lo_p;
    else {
        sure &= fast_edge(mu_p - (double)(ns * s_p), ep, lo_p);
        sure &= fast_edge(mu_p + (double)(ns * s_p), ep, hi_p);
    }
    if (!sure) return depo_window_f64(T0, X, Y, Z, Q, pp, d);
    const long long n_t = hi_t - lo_t + 1, n_p = hi_p - lo_p + 1;
    const long long lim = 1LL << 30;
    d.mu_t = d.mu_p = d.inv_t = d.inv_p = 0.f;
    d.q = 0.f;
    d.lo_t = d.lo_p = 0;
    d.nt = d.np = 0;
    if (n_t > WCT_MAX_WINDOW_TICKS || n_p > WCT_MAX_WINDOW_IMPACTS || lo_t < -lim || lo_t > lim || lo_p < -lim ||
        lo_p > lim)
        return false;
    d.lo_t = (int32_t)lo_t;
    d.lo_p = (int32_t)lo_p;
    d.nt = (int16_t)n_t;
    d.np = (int16_t)n_p;
    d.mu_t = (float)(mu_t - (double)lo_t);
    d.mu_p = (float)(mu_p - (double)lo_p);
    d.inv_t = dt ? 0.f : 0.70710678118654752f / s_t;
    d.inv_p = dp ? 0.f : 0.70710678118654752f / s_p;
    d.q = (float)Q;
    return true;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace wct
