// Noise addition and digitisation of the simulated waveforms: the steps after the
// convolution of §2 (the waveform becomes the ADC samples a readout would record).
//
// Per bin: v = gain * waveform + baseline + noise, code = floor(v + 1/2) clamped to
// [0, 2^bits - 1].  White noise: noise = noise_rms * z, z from the counter-based Philox stream,
// one call per four consecutive ticks of a wire, counter (tick / 4, wire, 0, (0x80 | plane) << 24
// | event), Box-Muller pairs for ticks 4k, 4k+1 and 4k+2, 4k+3.  Coloured noise: a noise
// waveform made beforehand from a per-plane amplitude spectrum (k_noise_spectrum, then the
// inverse row transform) is added instead.  The arithmetic is explicitly rounded FP32 (no
// contraction), so a host evaluation of the same float operations takes the same integer
// decision.
#include "wct_internal.cuh"
#include "wct_device.cuh"

namespace wct {

namespace {

__global__ void __launch_bounds__(256)
k_digitize(const float *__restrict__ wf, int16_t *__restrict__ adc, int n_wires, int n_ticks, AdcParams a,
           uint32_t c3) {
    const int n_quads = (n_ticks + 3) >> 2;
    const int64_t total = (int64_t)n_wires * n_quads;
    const bool vec = (n_ticks & 3) == 0 && (reinterpret_cast<uintptr_t>(wf) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(adc) & 7) == 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx / n_quads), qd = (int)(idx - (int64_t)w * n_quads);
        const int t0 = qd << 2;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (a.add_noise && !a.noise_wave) {
            const uint4 x = philox4x32_10_rk(make_uint4((uint32_t)qd, (uint32_t)w, 0u, c3), a.rk);
            const float2 p0 = box_muller(x.x, x.y), p1 = box_muller(x.z, x.w);
            z[0] = p0.x;
            z[1] = p0.y;
            z[2] = p1.x;
            z[3] = p1.y;
        }
        const size_t base = (size_t)w * n_ticks + t0;
        float v[4];
        if (vec) {
            const float4 f = *reinterpret_cast<const float4 *>(wf + base);
            v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
        } else {
#pragma unroll
            for (int l = 0; l < 4; ++l) v[l] = t0 + l < n_ticks ? wf[base + l] : 0.f;
        }
        float nz[4];
#pragma unroll
        for (int l = 0; l < 4; ++l)
            nz[l] = a.noise_wave ? (t0 + l < n_ticks ? a.noise_wave[base + l] : 0.f) : __fmul_rn(a.noise_rms, z[l]);
        int16_t c[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const float s = __fadd_rn(__fadd_rn(__fmul_rn(a.gain, v[l]), a.baseline), nz[l]);
            float code = floorf(__fadd_rn(s, 0.5f));
            code = fminf(fmaxf(code, 0.f), a.max_code);      // NaN -> 0 (fmaxf returns the number)
            c[l] = (int16_t)code;
        }
        if (vec) {
            short4 o;
            o.x = c[0], o.y = c[1], o.z = c[2], o.w = c[3];
            *reinterpret_cast<short4 *>(adc + base) = o;
        } else {
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (t0 + l < n_ticks) adc[base + l] = c[l];
        }
    }
}

// Coloured-noise spectrum of every wire: N[w][f] = scale * amp[f] * (z_re + i z_im) / sqrt(2),
// z from Philox at counter (f / 2, wire, 1, c3): words 0,1 give bin 2k, words 2,3 bin 2k+1
// (Box-Muller pairs); the DC and Nyquist (f = M) bins are real.  Bins from F up to the row
// stride are zero.  One thread per bin pair.
__global__ void __launch_bounds__(256)
k_noise_spectrum(const float *__restrict__ amp, int F, int M, int n_wires, int Fs, float scale, AdcParams a,
                 uint32_t c3, float2 *__restrict__ spec) {
    const int pairs = (Fs + 1) >> 1;
    const int64_t total = (int64_t)n_wires * pairs;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx / pairs), k = (int)(idx - (int64_t)w * pairs);
        const uint4 x = philox4x32_10_rk(make_uint4((uint32_t)k, (uint32_t)w, 1u, c3), a.rk);
        const float2 z0 = box_muller(x.x, x.y), z1 = box_muller(x.z, x.w);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int f = 2 * k + l;
            if (f >= Fs) break;
            float2 v = make_float2(0.f, 0.f);
            if (f < F) {
                const float2 z = l ? z1 : z0;
                const float s = scale * amp[f] * 0.70710678118654752f;
                v = make_float2(s * z.x, (f == 0 || f == M) ? 0.f : s * z.y);
            }
            spec[(size_t)w * Fs + f] = v;
        }
    }
}

}  // namespace

cudaError_t launch_noise_spectrum(const float *amp, int F, int M, int n_wires, int Fs, float scale, const AdcParams &a,
                                  uint32_t c3, float2 *spec, cudaStream_t s) {
    const int64_t total = (int64_t)n_wires * ((Fs + 1) >> 1);
    if (total <= 0) return cudaSuccess;
    const int64_t want = (total + 255) / 256;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    k_noise_spectrum<<<blocks, 256, 0, s>>>(amp, F, M, n_wires, Fs, scale, a, c3, spec);
    return cudaGetLastError();
}

cudaError_t launch_digitize(const float *wf, int16_t *adc, int n_wires, int n_ticks, const AdcParams &a, uint32_t c3,
                            cudaStream_t s) {
    const int64_t total = (int64_t)n_wires * ((n_ticks + 3) >> 2);
    if (total <= 0) return cudaSuccess;
    const int64_t want = (total + 255) / 256;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    k_digitize<<<blocks, 256, 0, s>>>(wf, adc, n_wires, n_ticks, a, c3);
    return cudaGetLastError();
}

}  // namespace wct
