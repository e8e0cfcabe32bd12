// Device-side helpers: Philox4x32-10, Box-Muller, integer floor division, status flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// Two standard normals from two 32-bit words: u = (x + 1/2) 2^-32 in (0,1),
// r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float s32 = 2.3283064365386963e-10f;   // 2^-32
    const float h32 = 1.1641532182693481e-10f;   // 2^-33
    const float ua = fmaf(__uint2float_rn(a), s32, h32);
    const float ub = fmaf(__uint2float_rn(b), s32, h32);
    const float r = sqrtf(fmaxf(-2.0f * logf(ua), 0.0f));
    float sn, cs;
    sincospif(2.0f * ub, &sn, &cs);
    return make_float2(r * cs, r * sn);
}

__device__ __forceinline__ int floor_div(int a, int b) {   // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace wct
