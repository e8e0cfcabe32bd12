// Convolution with the detector response (paper §2, step 3: "the main computation here is
// FFT").  The paper calls vendor FFT libraries (cuFFT / rocFFT / FFTW, §4.1); here the
// transforms are hand-written:
//
//   k_row_r2c   one CTA per wire row: real FFT along ticks of the zero-padded row (length
//               P = 2M, P >= n_ticks + n_resp_ticks - 1, 7-smooth), computed as a complex
//               FFT of length M of the even/odd-packed row in shared memory (mixed-radix
//               Stockham, radices 2,3,4,5,7,8, each stage staged through registers) plus the
//               usual split into the M + 1 half-spectrum bins.
//   k_wire_stage one thread per spectrum bin f and a run of wires: the convolution across
//               wires is a 21-tap complex stencil per time frequency,
//                   T[w, f] = sum_k S[w + 10 - k, f] * Rt[k, f],
//               where Rt[k, f] is the time-spectrum of response row k (scaled by 1/M).  It is
//               linear (zero outside the plane), so no FFT along wires and no 2D response
//               spectrum is needed.
//   k_row_c2r   one CTA per wire row: inverse of k_row_r2c, cropped to n_ticks.
#include "wct_internal.cuh"
#include "wct_device.cuh"
#include "wct_tma.cuh"

#include <algorithm>
#include <initializer_list>
#include <mutex>

namespace wct {

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// multiply by +i (INV) or -i (forward): the sign of the transform's exponent times i
template <bool INV>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---- small DFTs in registers: y_m = sum_n x_n exp(s 2 pi i n m / R), s = -1 forward ------
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = mul_si<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <bool INV>
struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        const float h = 0.7071067811865476f;
        const float sg = INV ? 1.f : -1.f;
        // twiddles exp(s 2 pi i k / 8), k = 1, 2, 3
        o[1] = cmul(o[1], make_float2(h, sg * h));
        o[2] = mul_si<INV>(o[2]);
        o[3] = cmul(o[3], make_float2(-h, sg * h));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// Odd R: pair x_n with x_{R-n}; y_m = x_0 + sum_n t_n cos(2 pi n m / R) + s i sum_n u_n sin(...)
template <int R>
struct OddTab;
template <>
struct OddTab<3> {
    __device__ __forceinline__ static float c(int k) { return -0.5f; }
    __device__ __forceinline__ static float s(int k) { return 0.8660254037844387f; }
};
template <>
struct OddTab<5> {
    __device__ __forceinline__ static float c(int k) { return k == 1 ? 0.30901699437494745f : -0.8090169943749473f; }
    __device__ __forceinline__ static float s(int k) { return k == 1 ? 0.9510565162951535f : 0.5877852522924732f; }
};
template <>
struct OddTab<7> {
    __device__ __forceinline__ static float c(int k) {
        return k == 1 ? 0.6234898018587336f : (k == 2 ? -0.22252093395631434f : -0.900968867902419f);
    }
    __device__ __forceinline__ static float s(int k) {
        return k == 1 ? 0.7818314824680298f : (k == 2 ? 0.9749279121818236f : 0.43388373911755823f);
    }
};

template <int R, bool INV>
struct DftOdd {
    __device__ __forceinline__ static void run(float2 *v) {
        constexpr int H = (R - 1) / 2;
        float2 t[H], u[H];
#pragma unroll
        for (int n = 1; n <= H; ++n) {
            t[n - 1] = cadd(v[n], v[R - n]);
            u[n - 1] = csub(v[n], v[R - n]);
        }
        float2 y0 = v[0];
#pragma unroll
        for (int n = 0; n < H; ++n) y0 = cadd(y0, t[n]);
        float2 out[R];
        out[0] = y0;
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            float2 a = v[0], b = make_float2(0.f, 0.f);
#pragma unroll
            for (int n = 1; n <= H; ++n) {
                const int k = (n * m) % R;                  // 1..R-1
                const int kk = k <= H ? k : R - k;         // cos symmetric, sin antisymmetric
                const float cs = OddTab<R>::c(kk);
                const float sn = k <= H ? OddTab<R>::s(kk) : -OddTab<R>::s(kk);
                a = fma2(t[n - 1], make_float2(cs, cs), a);
                b = fma2(u[n - 1], make_float2(sn, sn), b);
            }
            const float2 ib = mul_si<INV>(b);
            out[m] = cadd(a, ib);
            out[R - m] = csub(a, ib);
        }
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = out[m];
    }
};
template <bool INV>
struct Dft<3, INV> : DftOdd<3, INV> {};
template <bool INV>
struct Dft<5, INV> : DftOdd<5, INV> {};
template <bool INV>
struct Dft<7, INV> : DftOdd<7, INV> {};

// ---- compile-time roots of unity for the composite butterflies --------------------------
// Taylor series of sin / cos on [-pi, pi] (17 terms: the first omitted term is below 1e-19),
// evaluated by the compiler in double and rounded once to float.
__host__ __device__ constexpr double ct_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n <= 16; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n <= 16; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// exp(s 2 pi i m / R), s = -1 forward, +1 inverse; the angle is reduced to (-pi, pi] exactly
// through m mod R before it is formed
template <int R, int m, bool INV>
struct Root {
    static constexpr int mm = ((m % R) + R) % R;
    static constexpr int mr = 2 * mm > R ? mm - R : mm;
    static constexpr double a = 2.0 * 3.14159265358979323846 * (double)mr / (double)R;
    static constexpr float re = (float)ct_cos(a);
    static constexpr float im = (float)((INV ? 1.0 : -1.0) * ct_sin(a));
};

// Size R1 R2 DFT in registers by one Cooley-Tukey split: with r = r1 + R1 r2 and
// s = R2 s1 + s2, X[s] = sum_r1 w_R1^(r1 s1) [w_R^(r1 s2) sum_r2 v[r1 + R1 r2] w_R2^(r2 s2)]
// (w_n = exp(s 2 pi i / n)): R1 DFTs of size R2, the inner twiddles, R2 DFTs of size R1.
// Lets one Stockham pass through shared memory do the work of two.
template <int R1, int R2, bool INV>
struct DftComp {
    static constexpr int R = R1 * R2;
    template <int I>
    __device__ __forceinline__ static void twiddle(float2 (&y)[R1][R2]) {
        if constexpr (I < R) {
            constexpr int r1 = I / R2, s2 = I % R2;
            if constexpr (r1 > 0 && s2 > 0) {
                using W = Root<R, r1 * s2, INV>;
                y[r1][s2] = cmul(y[r1][s2], make_float2(W::re, W::im));
            }
            twiddle<I + 1>(y);
        }
    }
    __device__ __forceinline__ static void run(float2 *v) {
        float2 y[R1][R2];
#pragma unroll
        for (int r1 = 0; r1 < R1; ++r1) {
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) y[r1][r2] = v[r1 + R1 * r2];
            Dft<R2, INV>::run(y[r1]);
        }
        twiddle<0>(y);
#pragma unroll
        for (int s2 = 0; s2 < R2; ++s2) {
            float2 c[R1];
#pragma unroll
            for (int r1 = 0; r1 < R1; ++r1) c[r1] = y[r1][s2];
            Dft<R1, INV>::run(c);
#pragma unroll
            for (int s1 = 0; s1 < R1; ++s1) v[R2 * s1 + s2] = c[s1];
        }
    }
};
template <bool INV>
struct Dft<20, INV> : DftComp<4, 5, INV> {};
template <bool INV>
struct Dft<25, INV> : DftComp<5, 5, INV> {};
template <bool INV>
struct Dft<28, INV> : DftComp<4, 7, INV> {};
template <bool INV>
struct Dft<35, INV> : DftComp<5, 7, INV> {};

// R1 of a composite radix above (1 for a plain radix)
template <int R>
constexpr int inner_factor() {
    return (R == 20 || R == 28) ? 4 : (R == 25 || R == 35) ? 5 : 1;
}

// One Stockham stage of radix R, out of place (in -> out).  With Ns = product of the radices
// of the earlier stages, butterfly j (j < M/R) reads in[j + r M/R], applies the twiddles
// exp(s 2 pi i r (j mod Ns) / (Ns R)), does a size-R DFT and writes out[(j div Ns) Ns R +
// (j mod Ns) + r Ns].  One butterfly at a time per thread keeps register use at ~2R.
template <int R, bool INV>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ in, float2 *__restrict__ out, int M, int Ns,
                                          const float2 *__restrict__ tw) {
    const int nb = M / R;
    const int stride = M / (Ns * R);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * nb];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * k * stride];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        Dft<R, INV>::run(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
    }
    __syncthreads();
}

__device__ __forceinline__ int plan_radix(const FFTPlan &p, int s) { return (int)((p.radix_code >> (4 * s)) & 15u); }

// Stages [s_begin, s_end) of the complex FFT of length M in shared memory.  The first of them
// reads `src`; each stage writes whichever of x / y it is not reading.  tw is the
// exp(-2 pi i k / M) table (shared or global memory).  Returns the buffer holding the result.
template <bool INV>
__device__ const float2 *cta_fft_range(const float2 *src, float2 *x, float2 *y, const FFTPlan &p,
                                       const float2 *tw, int s_begin, int s_end) {
    int Ns = 1;
    for (int s = 0; s < s_begin; ++s) Ns *= plan_radix(p, s);
    const float2 *in = src;
    for (int s = s_begin; s < s_end; ++s) {
        const int R = plan_radix(p, s);
        float2 *out = (in == x) ? y : x;
        switch (R) {
            case 2: fft_stage<2, INV>(in, out, p.M, Ns, tw); break;
            case 3: fft_stage<3, INV>(in, out, p.M, Ns, tw); break;
            case 4: fft_stage<4, INV>(in, out, p.M, Ns, tw); break;
            case 5: fft_stage<5, INV>(in, out, p.M, Ns, tw); break;
            case 7: fft_stage<7, INV>(in, out, p.M, Ns, tw); break;
            default: fft_stage<8, INV>(in, out, p.M, Ns, tw); break;
        }
        in = out;
        Ns *= R;
    }
    return in;
}

// Complex FFT of length M in shared memory, ping-ponging between a and b.
template <bool INV>
__device__ const float2 *cta_fft(float2 *a, float2 *b, const FFTPlan &p) {
    return cta_fft_range<INV>(a, a, b, p, p.tw, 0, p.n_stages);
}

// ---- forward: real row -> half spectrum -------------------------------------------------
__global__ void __launch_bounds__(512)
k_row_r2c(FFTPlan p, const float *__restrict__ in, int64_t in_stride, int n_cols, float2 *__restrict__ spec) {
    extern __shared__ float2 smem2[];
    float2 *buf = smem2;
    const int M = p.M;
    const int row = blockIdx.x;
    const float *src = in + (int64_t)row * in_stride;
    const bool vec = ((in_stride & 1) == 0) && ((reinterpret_cast<uintptr_t>(in) & 7) == 0);
    for (int n = threadIdx.x; n < M; n += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (2 * n + 1 < n_cols) {
            v = vec ? reinterpret_cast<const float2 *>(src)[n] : make_float2(src[2 * n], src[2 * n + 1]);
        } else if (2 * n < n_cols) {
            v.x = src[2 * n];
        }
        buf[n] = v;
    }
    __syncthreads();
    const float2 *Z = cta_fft<false>(buf, smem2 + p.M, p);
    // X[k] = (Z[k] + conj Z[M-k]) / 2 - i exp(-2 pi i k / P) (Z[k] - conj Z[M-k]) / 2
    float2 *out = spec + (int64_t)row * p.Fs;
    for (int k = threadIdx.x; k < p.Fu; k += blockDim.x) {
        float2 X = make_float2(0.f, 0.f);
        if (k <= M) {
            const float2 a = Z[k == M ? 0 : k];
            const float2 b = conjf2(Z[k == 0 ? 0 : M - k]);
            const float2 wd = cmul(__ldg(&p.rtw[k]), csub(a, b));
            const float2 s = cadd(a, b);
            X = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
        }
        out[k] = X;
    }
}

// ---- inverse: half spectrum -> real row (cropped), unnormalised (scale lives in Rt) -----
__global__ void __launch_bounds__(512)
k_row_c2r(FFTPlan p, const float2 *__restrict__ spec, float *__restrict__ out, int64_t out_stride, int n_cols) {
    extern __shared__ float2 smem2[];
    float2 *buf = smem2;
    const int M = p.M;
    const int row = blockIdx.x;
    const float2 *X = spec + (int64_t)row * p.Fs;
    // E = (X[k] + conj X[M-k]) / 2, O = exp(2 pi i k / P) (X[k] - conj X[M-k]) / 2, Z = E + i O
    const float2 zero = make_float2(0.f, 0.f);
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const float2 a = k < p.Fu ? X[k] : zero;
        const float2 b = M - k < p.Fu ? conjf2(X[M - k]) : zero;
        const float2 O = cmul(conjf2(__ldg(&p.rtw[k])), csub(a, b));
        const float2 s = cadd(a, b);
        buf[k] = make_float2(0.5f * (s.x - O.y), 0.5f * (s.y + O.x));
    }
    __syncthreads();
    const float2 *z = cta_fft<true>(buf, smem2 + p.M, p);
    float *dst = out + (int64_t)row * out_stride;
    const bool vec = ((out_stride & 1) == 0) && ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
    for (int n = threadIdx.x; 2 * n < n_cols; n += blockDim.x) {
        const float2 v = z[n];
        if (2 * n + 1 < n_cols) {
            if (vec) {
                reinterpret_cast<float2 *>(dst)[n] = v;
            } else {
                dst[2 * n] = v.x;
                dst[2 * n + 1] = v.y;
            }
        } else {
            dst[2 * n] = v.x;
        }
    }
}

constexpr int kRowThreadsCt = 1024;

// ---- compile-time radix plans ---------------------------------------------------------
// For the common lengths the radix sequence is a template parameter: every stage's Ns, stride
// and butterfly count are constants, so the index arithmetic needs no runtime division and
// the per-thread butterfly loop unrolls.  Same Stockham stage as fft_stage.
template <int R, int NS, int M, int T, bool INV>
__device__ __forceinline__ void stage_ct(const float2 *__restrict__ in, float2 *__restrict__ out,
                                         const float2 *__restrict__ tw) {
    constexpr int NB = M / R;
    constexpr int STRIDE = M / (NS * R);
    constexpr int ITER = (NB + T - 1) / T;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int j = threadIdx.x + it * T;
        if (ITER * T == NB || j < NB) {
            const int k = j % NS;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = in[j + r * NB];
            if (NS > 1) {
                float2 w1 = tw[k * STRIDE];
                if (INV) w1.y = -w1.y;
                float2 w = w1;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    v[r] = cmul(v[r], w);
                    if (r + 1 < R) w = cmul(w, w1);
                }
            }
            Dft<R, INV>::run(v);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) out[base + r * NS] = v[r];
        }
    }
    __syncthreads();
}

template <int M, int T, bool INV, int NS, int R, int... Rest>
struct FftCt {
    __device__ __forceinline__ static const float2 *run(const float2 *in, float2 *x, float2 *y, const float2 *tw) {
        float2 *out = (in == x) ? y : x;
        stage_ct<R, NS, M, T, INV>(in, out, tw);
        if constexpr (sizeof...(Rest) == 0) return out;
        else return FftCt<M, T, INV, NS * R, Rest...>::run(out, x, y, tw);
    }
};

template <int... Rs>
struct CtPlan {
    static constexpr int M = (Rs * ...);
};

// Policy used by the persistent kernels: stages [s0, s1) with s0 / s1 in {0, 1, n}.
struct RuntimeFft {
    template <bool INV>
    __device__ __forceinline__ static const float2 *range(const float2 *src, float2 *x, float2 *y, const FFTPlan &p,
                                                          const float2 *tw, int s0, int s1) {
        return cta_fft_range<INV>(src, x, y, p, tw, s0, s1);
    }
};

template <class Plan>
struct CompiledFft;

template <int R0, int... Rs>
struct CompiledFft<CtPlan<R0, Rs...>> {
    static constexpr int M = CtPlan<R0, Rs...>::M;
    template <bool INV>
    __device__ __forceinline__ static const float2 *range(const float2 *src, float2 *x, float2 *y, const FFTPlan &,
                                                          const float2 *tw, int s0, int s1) {
        if (s0 == 0 && s1 == 1) return FftCt<M, kRowThreadsCt, INV, 1, R0>::run(src, x, y, tw);
        if (s0 == 1) {
            if constexpr (sizeof...(Rs) > 0) return FftCt<M, kRowThreadsCt, INV, R0, Rs...>::run(src, x, y, tw);
            else return src;
        }
        return FftCt<M, kRowThreadsCt, INV, 1, R0, Rs...>::run(src, x, y, tw);
    }
};

// ---- register-staged row transforms: small CTAs, whole row in one shared buffer ---------
// One 128-thread CTA per row; each thread keeps all its butterflies of a stage in registers
// (about M / 128 points), so a stage is: load everything, barrier, arithmetic, store in place,
// barrier.  Several CTAs share an SM (one M-point buffer each, ~39 KB at M = 4900), so one
// CTA's global loads overlap the others' arithmetic; twiddles come from the global table
// through L1.
constexpr int kRsThreads = 128;

template <int R, int NS, int M, bool INV>
__device__ __forceinline__ void stage_rs(float2 *buf, const float2 *__restrict__ tw) {
    constexpr int NB = M / R;
    constexpr int STRIDE = M / (NS * R);
    constexpr int ITER = (NB + kRsThreads - 1) / kRsThreads;
    float2 v[ITER][R];
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int j = threadIdx.x + it * kRsThreads;
        if (ITER * kRsThreads == NB || j < NB) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[it][r] = buf[j + r * NB];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int j = threadIdx.x + it * kRsThreads;
        if (ITER * kRsThreads == NB || j < NB) {
            const int k = j % NS;
            if (NS > 1) {
                // one table load per butterfly; the higher twiddles are its powers
                float2 w1 = __ldg(&tw[k * STRIDE]);
                if (INV) w1.y = -w1.y;
                float2 w = w1;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    v[it][r] = cmul(v[it][r], w);
                    if (r + 1 < R) w = cmul(w, w1);
                }
            }
            Dft<R, INV>::run(v[it]);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[base + r * NS] = v[it][r];
        }
    }
    __syncthreads();
}

template <int M, bool INV, int NS, int R, int... Rest>
__device__ __forceinline__ void fft_rs(float2 *buf, const float2 *tw) {
    stage_rs<R, NS, M, INV>(buf, tw);
    if constexpr (sizeof...(Rest) > 0) fft_rs<M, INV, NS * R, Rest...>(buf, tw);
}

template <class Plan>
struct RsFft;
template <int... Rs>
struct RsFft<CtPlan<Rs...>> {
    static constexpr int M = CtPlan<Rs...>::M;
    template <bool INV>
    __device__ __forceinline__ static void run(float2 *buf, const float2 *tw) {
        fft_rs<M, INV, 1, Rs...>(buf, tw);
    }
};

template <class Plan>
__global__ void __launch_bounds__(kRsThreads, 5)
k_row_r2c_rs(FFTPlan p, const float *__restrict__ in, int n_cols, float2 *__restrict__ spec) {
    extern __shared__ float2 buf[];
    constexpr int M = RsFft<Plan>::M;
    const int row = blockIdx.x;
    const float4 *src = reinterpret_cast<const float4 *>(in + (size_t)row * n_cols);   // n_cols % 4 == 0
    const int q4 = n_cols >> 2;
    for (int i = threadIdx.x; i < q4; i += kRsThreads) {
        const float4 v = src[i];
        buf[2 * i] = make_float2(v.x, v.y);
        buf[2 * i + 1] = make_float2(v.z, v.w);
    }
    for (int k = 2 * q4 + threadIdx.x; k < M; k += kRsThreads) buf[k] = make_float2(0.f, 0.f);
    __syncthreads();
    RsFft<Plan>::template run<false>(buf, p.tw);
    float2 *out = spec + (size_t)row * p.Fs;
    for (int k = threadIdx.x; k < p.Fu; k += kRsThreads) {
        float2 X = make_float2(0.f, 0.f);
        if (k <= M) {
            const float2 a = buf[k == M ? 0 : k];
            const float2 b = conjf2(buf[k == 0 ? 0 : M - k]);
            const float2 wd = cmul(__ldg(&p.rtw[k]), csub(a, b));
            const float2 sm = cadd(a, b);
            X = make_float2(0.5f * (sm.x + wd.y), 0.5f * (sm.y - wd.x));
        }
        out[k] = X;
    }
}

template <class Plan>
__global__ void __launch_bounds__(kRsThreads, 5)
k_row_c2r_rs(FFTPlan p, const float2 *__restrict__ spec, float *__restrict__ out, int n_cols) {
    extern __shared__ float2 buf[];
    constexpr int M = RsFft<Plan>::M;
    const int row = blockIdx.x;
    const float2 *X = spec + (size_t)row * p.Fs;
    const float2 zero = make_float2(0.f, 0.f);
    for (int k = threadIdx.x; k < M; k += kRsThreads) {
        const float2 a = k < p.Fu ? X[k] : zero;
        const float2 b = M - k < p.Fu ? conjf2(X[M - k]) : zero;
        const float2 O = cmul(conjf2(__ldg(&p.rtw[k])), csub(a, b));
        const float2 sm = cadd(a, b);
        buf[k] = make_float2(0.5f * (sm.x - O.y), 0.5f * (sm.y + O.x));
    }
    __syncthreads();
    RsFft<Plan>::template run<true>(buf, p.tw);
    float4 *dst = reinterpret_cast<float4 *>(out + (size_t)row * n_cols);             // n_cols % 4 == 0
    const int q4 = n_cols >> 2;
    for (int i = threadIdx.x; i < q4; i += kRsThreads) {
        const float2 a = buf[2 * i], b = buf[2 * i + 1];
        dst[i] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// ---- persistent row transforms: one CTA per SM, rows streamed in by bulk copies ---------
// Shared memory: A (staging row, M + 2 entries), B, C (ping-pong, M each), TW (M twiddles),
// RTW (M + 1 real-split twiddles, padded to M + 2), one mbarrier.  The twiddle tables are
// loaded once per CTA.  While the transform of row r runs on B / C, the bulk copy of row
// r + gridDim.x lands in A.
constexpr int kRowThreads = 1024;

size_t row_tma_smem_bytes(int M) { return sizeof(float2) * (5 * (size_t)M + 4) + 16; }

struct RowSmem {
    float2 *A, *B, *C, *TW, *RTW;
    uint64_t *bar;
    __device__ __forceinline__ RowSmem(float4 *base, int M) {
        A = reinterpret_cast<float2 *>(base);
        B = A + M + 2;
        C = B + M;
        TW = C + M;
        RTW = TW + M;
        bar = reinterpret_cast<uint64_t *>(RTW + M + 2);
    }
};

__device__ __forceinline__ void row_tma_init(const FFTPlan &p, float2 *TW, float2 *RTW, uint64_t *bar) {
    for (int k = threadIdx.x; k < p.M; k += blockDim.x) TW[k] = p.tw[k];
    for (int k = threadIdx.x; k <= p.M; k += blockDim.x) RTW[k] = p.rtw[k];
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
}

// All threads wait for the row; if any thread's bounded wait ran out, thread 0 records the
// timeout, waits once more (bounded) for the copy in flight, and every thread leaves.
__device__ __forceinline__ bool row_tma_wait(uint64_t *bar, uint32_t parity, int32_t *status) {
    const bool ok = mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            set_status(status, ST_ETIMEOUT);
            mbar_wait(bar, parity);
        }
        return false;
    }
    return true;
}

template <class FFT>
__global__ void __launch_bounds__(kRowThreads, 1)
k_row_r2c_tma(FFTPlan p, const float *__restrict__ in, int n_rows, int n_cols, float2 *__restrict__ spec,
              int32_t *status) {
    extern __shared__ float4 sm4[];
    const int M = p.M;
    const RowSmem L(sm4, M);
    float2 *A = L.A, *B = L.B, *C = L.C, *TW = L.TW, *RTW = L.RTW;
    uint64_t *bar = L.bar;
    const int half = n_cols >> 1;                      // n_cols % 4 == 0
    const uint32_t bytes = (uint32_t)n_cols * 4u;
    row_tma_init(p, TW, RTW, bar);
    for (int k = half + threadIdx.x; k < M + 2; k += blockDim.x) A[k] = make_float2(0.f, 0.f);   // zero pad, kept
    __syncthreads();
    int row = blockIdx.x;
    if (threadIdx.x == 0 && row < n_rows) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(A, in + (size_t)row * n_cols, bytes, bar);
    }
    uint32_t parity = 0;
    for (; row < n_rows; row += gridDim.x) {
        if (!row_tma_wait(bar, parity, status)) return;
        parity ^= 1u;
        FFT::template range<false>(A, B, C, p, TW, 0, 1);    // A -> B, ends with a CTA barrier
        const int next = row + gridDim.x;
        if (threadIdx.x == 0 && next < n_rows) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(A, in + (size_t)next * n_cols, bytes, bar);
        }
        const float2 *Z = FFT::template range<false>(B, B, C, p, TW, 1, p.n_stages);
        float2 *out = spec + (size_t)row * p.Fs;
        for (int k = threadIdx.x; k < p.Fu; k += blockDim.x) {
            float2 X = make_float2(0.f, 0.f);
            if (k <= M) {
                const float2 a = Z[k == M ? 0 : k];
                const float2 b = conjf2(Z[k == 0 ? 0 : M - k]);
                const float2 wd = cmul(RTW[k], csub(a, b));
                const float2 sm = cadd(a, b);
                X = make_float2(0.5f * (sm.x + wd.y), 0.5f * (sm.y - wd.x));
            }
            out[k] = X;
        }
        __syncthreads();
    }
}

template <class FFT>
__global__ void __launch_bounds__(kRowThreads, 1)
k_row_c2r_tma(FFTPlan p, const float2 *__restrict__ spec, int n_rows, float *__restrict__ out, int n_cols,
              int32_t *status) {
    extern __shared__ float4 sm4[];
    const int M = p.M;
    const RowSmem L(sm4, M);
    float2 *A = L.A, *B = L.B, *C = L.C, *TW = L.TW, *RTW = L.RTW;
    uint64_t *bar = L.bar;
    const uint32_t bytes = (uint32_t)p.Fu * 8u;        // Fu <= Fs <= M + 2
    row_tma_init(p, TW, RTW, bar);
    for (int k = p.Fu + threadIdx.x; k < M + 2; k += blockDim.x) A[k] = make_float2(0.f, 0.f);   // kept
    __syncthreads();
    int row = blockIdx.x;
    if (threadIdx.x == 0 && row < n_rows) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(A, spec + (size_t)row * p.Fs, bytes, bar);
    }
    uint32_t parity = 0;
    for (; row < n_rows; row += gridDim.x) {
        if (!row_tma_wait(bar, parity, status)) return;
        parity ^= 1u;
        // Z[k] = E + i O, E = (X[k] + conj X[M-k]) / 2, O = exp(2 pi i k / P)(X[k] - conj X[M-k]) / 2
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            const float2 a = A[k];
            const float2 b = conjf2(A[M - k]);
            const float2 O = cmul(conjf2(RTW[k]), csub(a, b));
            const float2 sm = cadd(a, b);
            B[k] = make_float2(0.5f * (sm.x - O.y), 0.5f * (sm.y + O.x));
        }
        __syncthreads();
        const int next = row + gridDim.x;
        if (threadIdx.x == 0 && next < n_rows) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(A, spec + (size_t)next * p.Fs, bytes, bar);
        }
        const float2 *z = FFT::template range<true>(B, B, C, p, TW, 0, p.n_stages);
        float *dst = out + (size_t)row * n_cols;
        for (int n2 = threadIdx.x; 2 * n2 < n_cols; n2 += blockDim.x) reinterpret_cast<float2 *>(dst)[n2] = z[n2];
        __syncthreads();
    }
}

// ---- paired row transforms: two persistent CTAs per SM -----------------------------------
// Shared memory per CTA: A and B (M + 2 entries each, ping-pong), TWH (the twiddles
// exp(-2 pi i k / M) for k <= M/2; the upper half follows from tw[M - k] = conj tw[k]) and
// one mbarrier: about 96 KB at M = 4900, so two CTAs share an SM and one CTA's barriers and
// copy waits overlap the other's arithmetic.  The real-split twiddles exp(-i pi k / M) are
// derived from the same table: tw[k / 2] for even k, tw[(k - 1) / 2] * exp(-i pi / M) for odd
// k.  The row copy lands in A; the transform runs A -> B -> A ...; for an odd stage count A is
// free after the last stage, so the next row's copy overlaps the output pass.
constexpr int kPairThreads = 512;
constexpr int kPairThreadsComposite = 256;

size_t row_pair_smem_bytes(int M) { return sizeof(float2) * (2 * (size_t)(M + 2) + (size_t)(M / 2 + 2)) + 16; }

struct PairSmem {
    float2 *A, *B, *TWH;
    uint64_t *bar;
    __device__ __forceinline__ PairSmem(float4 *base, int M) {
        A = reinterpret_cast<float2 *>(base);
        B = A + M + 2;
        TWH = B + M + 2;
        bar = reinterpret_cast<uint64_t *>(TWH + M / 2 + 2);
    }
};

template <int M>
__device__ __forceinline__ float2 tw_half(const float2 *TWH, int idx) {   // exp(-2 pi i idx / M), 0 <= idx < M
    const bool hi = idx > M / 2;
    float2 w = TWH[hi ? M - idx : idx];
    if (hi) w.y = -w.y;
    return w;
}

template <int M>
__device__ __forceinline__ float2 rtw_half(const float2 *TWH, float2 c1, int k) {   // exp(-i pi k / M), 0 <= k <= M
    const float2 w = tw_half<M>(TWH, k >> 1);
    return (k & 1) ? cmul(w, c1) : w;
}

// v[r] *= w1^r, r = 1 .. R - 1 (the Stockham input twiddles of one butterfly)
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[R], float2 w1) {
    constexpr int C = inner_factor<R>();
    if constexpr (C > 1) {
        // composite radix: w^(r1 + C r2) = w^r1 (w^C)^r2, two short power chains
        float2 pw[C];
        pw[1] = w1;
#pragma unroll
        for (int c = 2; c < C; ++c) pw[c] = cmul(pw[c - 1], w1);
        const float2 WC = cmul(pw[C - 1], w1);
#pragma unroll
        for (int c = 1; c < C; ++c) v[c] = cmul(v[c], pw[c]);
        float2 Q = WC;
#pragma unroll
        for (int r2 = 1; r2 < R / C; ++r2) {
            v[C * r2] = cmul(v[C * r2], Q);
#pragma unroll
            for (int c = 1; c < C; ++c) v[c + C * r2] = cmul(v[c + C * r2], cmul(pw[c], Q));
            if (r2 + 1 < R / C) Q = cmul(Q, WC);
        }
    } else {
        float2 w = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            v[r] = cmul(v[r], w);
            if (r + 1 < R) w = cmul(w, w1);
        }
    }
}

// Butterfly j of a Stockham stage (radix R after stages of product NS): loads its R inputs
// in[j + r M/R], applies the twiddles and the size-R DFT, leaving the outputs in v (output r
// belongs at (j - j mod NS) R + j mod NS + r NS).
template <int R, int NS, int M, bool INV>
__device__ __forceinline__ void butterfly(const float2 *__restrict__ in, const float2 *__restrict__ TWH, int j,
                                          float2 (&v)[R]) {
    constexpr int NB = M / R;
    constexpr int STRIDE = M / (NS * R);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * NB];
    if constexpr (NS > 1) {
        float2 w1 = tw_half<M>(TWH, (j % NS) * STRIDE);
        if (INV) w1.y = -w1.y;
        apply_twiddles<R>(v, w1);
    }
    Dft<R, INV>::run(v);
}

template <int R, int NS, int M, int T, bool INV>
__device__ __forceinline__ void stage_pair(const float2 *__restrict__ in, float2 *__restrict__ out,
                                           const float2 *__restrict__ TWH) {
    constexpr int NB = M / R;
    constexpr int ITER = (NB + T - 1) / T;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int j = threadIdx.x + it * T;
        if (ITER * T == NB || j < NB) {
            const int k = j % NS;
            float2 v[R];
            butterfly<R, NS, M, INV>(in, TWH, j, v);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) out[base + r * NS] = v[r];
        }
    }
    __syncthreads();
}

template <int M, int T, bool INV, int NS, int R, int... Rest>
struct FftPair {
    // stages from `in` (A or B) alternating between A and B; returns the buffer with the result
    __device__ __forceinline__ static float2 *run(float2 *in, float2 *A, float2 *B, const float2 *TWH) {
        float2 *out = (in == A) ? B : A;
        stage_pair<R, NS, M, T, INV>(in, out, TWH);
        if constexpr (sizeof...(Rest) == 0) return out;
        else return FftPair<M, T, INV, NS * R, Rest...>::run(out, A, B, TWH);
    }
};

template <int M>
__device__ __forceinline__ void pair_init(const FFTPlan &p, float2 *TWH, uint64_t *bar) {
    for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) TWH[k] = p.tw[k];
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
}

// generic-proxy writes of every thread to A are ordered before the next bulk copy into A
__device__ __forceinline__ void release_to_copy() {
    fence_proxy_async_smem();
    __syncthreads();
}

template <int T, int... Rs>
__global__ void __launch_bounds__(T, 2)
k_row_r2c_pair(FFTPlan p, const float *__restrict__ in, int n_rows, int n_cols, float2 *__restrict__ spec,
               int32_t *status, const uint8_t *__restrict__ act) {
    constexpr int M = (Rs * ...);
    constexpr bool kOdd = (sizeof...(Rs) & 1) != 0;     // result in B, A free after the last stage
    extern __shared__ float4 sm4[];
    const PairSmem L(sm4, M);
    float2 *A = L.A, *B = L.B;
    const float2 *TWH = L.TWH;
    uint64_t *bar = L.bar;
    const int half = n_cols >> 1;                      // n_cols % 4 == 0, half <= M
    const uint32_t bytes = (uint32_t)n_cols * 4u;
    const float2 c1 = p.rtw[1];
    pair_init<M>(p, L.TWH, bar);
    __syncthreads();
    // rows known to be all zero (act[row] == 0) are skipped: their spectra are never read
    auto next_row = [&](int r) {
        if (act)
            while (r < n_rows && !act[r]) r += gridDim.x;
        return r;
    };
    int row = next_row(blockIdx.x);
    if (threadIdx.x == 0 && row < n_rows) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(A, in + (size_t)row * n_cols, bytes, bar);
    }
    uint32_t parity = 0;
    for (int next; row < n_rows; row = next) {
        for (int k = half + threadIdx.x; k < M; k += T) A[k] = make_float2(0.f, 0.f);   // zero pad
        if (!row_tma_wait(bar, parity, status)) return;
        parity ^= 1u;
        const float2 *Z = FftPair<M, T, false, 1, Rs...>::run(A, A, B, TWH);
        next = next_row(row + gridDim.x);
        if constexpr (kOdd) {
            release_to_copy();
            if (threadIdx.x == 0 && next < n_rows) {
                mbar_arrive_expect_tx(bar, bytes);
                bulk_g2s(A, in + (size_t)next * n_cols, bytes, bar);
            }
        }
        float2 *out = spec + (size_t)row * p.Fs;
        for (int k = threadIdx.x; k < p.Fu; k += T) {
            float2 X = make_float2(0.f, 0.f);
            if (k <= M) {
                const float2 a = Z[k == M ? 0 : k];
                const float2 b = conjf2(Z[k == 0 ? 0 : M - k]);
                const float2 wd = cmul(rtw_half<M>(TWH, c1, k), csub(a, b));
                const float2 sm = cadd(a, b);
                X = make_float2(0.5f * (sm.x + wd.y), 0.5f * (sm.y - wd.x));
            }
            out[k] = X;
        }
        if constexpr (kOdd) {
            __syncthreads();                           // Z (in B) read before the next row writes B
        } else {
            release_to_copy();                         // Z (in A) read before the next copy into A
            if (threadIdx.x == 0 && next < n_rows) {
                mbar_arrive_expect_tx(bar, bytes);
                bulk_g2s(A, in + (size_t)next * n_cols, bytes, bar);
            }
        }
    }
}

template <int T, int... Rs>
__global__ void __launch_bounds__(T, 2)
k_row_c2r_pair(FFTPlan p, const float2 *__restrict__ spec, int n_rows, float *__restrict__ out, int n_cols,
               int32_t *status, const uint8_t *__restrict__ act) {
    constexpr int M = (Rs * ...);
    constexpr bool kOdd = (sizeof...(Rs) & 1) != 0;
    extern __shared__ float4 sm4[];
    const PairSmem L(sm4, M);
    float2 *A = L.A, *B = L.B;
    const float2 *TWH = L.TWH;
    uint64_t *bar = L.bar;
    const int Fu = p.Fu;                               // bins >= Fu are zero
    const uint32_t bytes = (uint32_t)Fu * 8u;          // Fu <= M + 2
    const float2 c1 = p.rtw[1];
    pair_init<M>(p, L.TWH, bar);
    __syncthreads();
    const float2 zero = make_float2(0.f, 0.f);
    // output rows known to be zero (act[row] == 0: no charge within the response's reach) are
    // written as zeros, without a copy or a transform
    auto next_row = [&](int r) {
        if (act)
            while (r < n_rows && !act[r]) {
                float2 *dz = reinterpret_cast<float2 *>(out + (size_t)r * n_cols);
                for (int n2 = threadIdx.x; 2 * n2 < n_cols; n2 += T) dz[n2] = zero;
                r += gridDim.x;
            }
        return r;
    };
    int row = next_row(blockIdx.x);
    if (threadIdx.x == 0 && row < n_rows) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(A, spec + (size_t)row * p.Fs, bytes, bar);
    }
    uint32_t parity = 0;
    for (int next; row < n_rows; row = next) {
        if (!row_tma_wait(bar, parity, status)) return;
        parity ^= 1u;
        // Z[k] = E + i O, E = (X[k] + conj X[M-k]) / 2, O = exp(2 pi i k / P)(X[k] - conj X[M-k]) / 2,
        // in place: one thread forms Z[k] and Z[M-k] from X[k] and X[M-k]; exp(-i pi (M-k) / M)
        // = -conj exp(-i pi k / M)
        for (int k = threadIdx.x; 2 * k <= M; k += T) {
            const int k2 = M - k;
            const float2 xk = k < Fu ? A[k] : zero;
            const float2 xm = k2 < Fu ? A[k2] : zero;
            const float2 r = rtw_half<M>(TWH, c1, k);
            {
                const float2 a = xk, b = conjf2(xm);
                const float2 O = cmul(conjf2(r), csub(a, b));
                const float2 sm = cadd(a, b);
                A[k] = make_float2(0.5f * (sm.x - O.y), 0.5f * (sm.y + O.x));
            }
            if (k > 0 && k2 != k) {
                const float2 a = xm, b = conjf2(xk);
                const float2 O = cmul(make_float2(-r.x, -r.y), csub(a, b));   // conj(-conj r) = -r
                const float2 sm = cadd(a, b);
                A[k2] = make_float2(0.5f * (sm.x - O.y), 0.5f * (sm.y + O.x));
            }
        }
        __syncthreads();
        const float2 *z = FftPair<M, T, true, 1, Rs...>::run(A, A, B, TWH);
        next = next_row(row + gridDim.x);
        if constexpr (kOdd) {
            release_to_copy();
            if (threadIdx.x == 0 && next < n_rows) {
                mbar_arrive_expect_tx(bar, bytes);
                bulk_g2s(A, spec + (size_t)next * p.Fs, bytes, bar);
            }
        }
        float *dst = out + (size_t)row * n_cols;
        for (int n2 = threadIdx.x; 2 * n2 < n_cols; n2 += T) reinterpret_cast<float2 *>(dst)[n2] = z[n2];
        if constexpr (kOdd) {
            __syncthreads();
        } else {
            release_to_copy();
            if (threadIdx.x == 0 && next < n_rows) {
                mbar_arrive_expect_tx(bar, bytes);
                bulk_g2s(A, spec + (size_t)next * p.Fs, bytes, bar);
            }
        }
    }
}

// ---- wire stage: 21-tap complex stencil across wires per frequency ----------------------
constexpr int KW = WCT_MAX_RESPONSE_WIRES;   // 21
constexpr int KC = KW / 2;                   // 10
constexpr int kStageThreads = 128;
constexpr int kStageRun = 64;                // wires per thread

__global__ void __launch_bounds__(kStageThreads)
k_wire_stage(const float2 *__restrict__ S, const float2 *__restrict__ Rt, int Fs, int Fu, int n_wires,
             float2 *__restrict__ T, int accumulate) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= Fu) return;
    const int w0 = blockIdx.y * kStageRun;
    const int w1 = min(w0 + kStageRun, n_wires);
    const int n_in = (w1 - w0) + 2 * KC;
    float2 r[KW], acc[KW];
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        r[k] = Rt[(int64_t)k * Fs + f];
        acc[k] = make_float2(0.f, 0.f);
    }
    // Input row s = w0 - KC + m contributes S[s] * Rt[k] to output w = s - KC + k, i.e. output
    // index i = m - 2 KC + k, kept in accumulator slot i mod KW; output i is complete once
    // m = i + 2 KC (k = 0) has been added.
    for (int mb = 0; mb < n_in; mb += KW) {
#pragma unroll
        for (int u = 0; u < KW; ++u) {
            const int m = mb + u;
            if (m < n_in) {
                const int s = w0 - KC + m;
                float2 x = make_float2(0.f, 0.f);
                if (s >= 0 && s < n_wires) x = S[(int64_t)s * Fs + f];
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const int slot = (u + 1 + k) % KW;
                    acc[slot].x = fmaf(x.x, r[k].x, fmaf(-x.y, r[k].y, acc[slot].x));
                    acc[slot].y = fmaf(x.x, r[k].y, fmaf(x.y, r[k].x, acc[slot].y));
                }
                const int done = (u + 1) % KW;
                if (m >= 2 * KC) {
                    float2 *dst = &T[(int64_t)(w0 + m - 2 * KC) * Fs + f];
                    *dst = accumulate ? cadd(acc[done], *dst) : acc[done];
                }
                acc[done] = make_float2(0.f, 0.f);
            }
        }
    }
}

// the tile clearing for the fallback wire stage, which does not take it as a side job
__global__ void __launch_bounds__(256) k_clear_tiles_fft(const ClearJob job) {
    clear_listed_tiles(job, blockIdx.x, gridDim.x, 256);
}

// ---- wire stage fed by bulk copies -------------------------------------------------------
// CTA = kStageFB consecutive frequencies x a run of wires_per_cta output wires.  The input rows
// s = w0 - KC + m (m = 0 .. n_out + 2 KC - 1) of the CTA's frequency slice (kStageFB complex =
// 1 KB per row) stream through a ring of kRingGroups groups of kGroupRows rows in shared memory,
// one mbarrier pair per group: full[g] completes when the group's copies landed, empty[g] when
// every consumer has taken its rows.  Group k holds the rows m = 8k - 4 .. 8k + 3, so the 8 rows
// that a block of 8 outputs adds to its window (rows 8q + 20 .. 8q + 27 for outputs 8q .. 8q + 7)
// are exactly group q + 3: a consumer does one wait, eight constant-offset loads and one release
// per block, with no per-row index arithmetic.  Rows outside the plane, and rows the forward
// transform skipped as all zero (act), are copied from a zero row, so the consumers never test
// them.  A producer thread issues the copies; the consumer
// threads (one per frequency) keep a window of 28 input rows in registers and run the 21-tap
// stencil in pull form, each input row read from shared memory once.
constexpr int kStageFB = 128;
constexpr int kStageWiresMax = 512;      // output wires per CTA at most (chosen at launch)
constexpr int kGroupRows = 8;
constexpr int kRingGroups = 4;
constexpr int kGroupLead = 3;            // groups loaded before the first block's: rows -4 .. 19
constexpr int kImpactWires = 32;         // output wires per CTA with several phases (shared tile)

// A frequency slice of zeros: the copy source of the rows outside the plane.
__device__ __align__(16) float2 g_zero_row[kStageFB] = {};

__global__ void __launch_bounds__(kStageFB + 32, 3)
k_wire_stage_tma(const float2 *__restrict__ S, const float2 *__restrict__ Rt, int Fs, int Fu, int n_wires,
                 int wires_per_cta, float2 *__restrict__ T, int32_t *status, const ClearJob clear, int accumulate,
                 int n_phases, int64_t s_phase_stride, int64_t r_phase_stride, const uint8_t *__restrict__ act) {
    __shared__ __align__(16) float2 ring[kRingGroups * kGroupRows][kStageFB];
    // impact mode (n_phases > 1): the CTA's outputs summed over the phases in shared memory
    // ([output wire][frequency], dynamic, wires_per_cta rows) and written to T once
    extern __shared__ float2 tile[];
    __shared__ uint64_t full[kRingGroups], empty[kRingGroups];
    __shared__ int s_issued, s_prod_done;               // groups the producer issued; it has stopped
    const int tid = threadIdx.x;
    const int f0 = blockIdx.x * kStageFB;
    const int nf = min(kStageFB, Fu - f0);             // even (Fu even, f0 multiple of 128)
    const uint32_t row_bytes = (uint32_t)nf * 8u;
    const int w0 = blockIdx.y * wires_per_cta;
    const int n_out = min(wires_per_cta, n_wires - w0);
    const int n_blocks = (n_out + kGroupRows - 1) / kGroupRows;
    const int n_groups = n_blocks + kGroupLead;         // groups of one phase
    if (tid == 0) {
        for (int i = 0; i < kRingGroups; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kStageFB);
        }
        s_issued = 0;
        s_prod_done = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid >= kStageFB) {
        // producer: lane 0 of the extra warp issues the copies group by group
        // (impact mode: the groups of every phase in turn, one ring sequence)
        if (tid == kStageFB) {
            for (int gg = 0; gg < n_phases * n_groups; ++gg) {
                const int ph = gg / n_groups, k = gg - ph * n_groups;
                const int gs = gg % kRingGroups, use = gg / kRingGroups;
                if (use > 0 && !mbar_wait(&empty[gs], (use - 1) & 1)) {
                    set_status(status, ST_ETIMEOUT);
                    break;
                }
                const float2 *Sp = S + (size_t)ph * s_phase_stride;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[gs], row_bytes * (uint32_t)kGroupRows);
                bool live_row[kGroupRows];
#pragma unroll
                for (int i = 0; i < kGroupRows; ++i) {
                    const int src_row = w0 - KC + kGroupRows * k - 4 + i;
                    live_row[i] = src_row >= 0 && src_row < n_wires && (!act || act[ph * n_wires + src_row]);
                }
#pragma unroll
                for (int i = 0; i < kGroupRows; ++i) {
                    const int src_row = w0 - KC + kGroupRows * k - 4 + i;
                    const float2 *src = live_row[i] ? Sp + (size_t)src_row * Fs + f0 : g_zero_row;
                    bulk_g2s(ring[gs * kGroupRows + i], src, row_bytes, &full[gs]);
                }
                *(volatile int *)&s_issued = gg + 1;
            }
            __threadfence_block();
            *(volatile int *)&s_prod_done = 1;
        }
        return;
    }
    // side job: clear this CTA's share of the grid tiles listed by the rasterizer (the grid
    // was read by the forward transform before this launch); consumers only
    if (clear.grid)
        clear_listed_tiles(clear, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y, kStageFB);
    const int f = f0 + tid;
    const bool live = tid < nf;
    constexpr int kOutBlock = kGroupRows;
    constexpr int kWin = kOutBlock + 2 * KC;           // rows 8q .. 8q + 27 of block q
    float2 rr[KW], ri[KW];                             // (re, re) and (im, im) of each tap
    bool ok = true;
    int g_fail = 0;                                    // first group whose wait ran out (if !ok)
    // the 8 rows of ring group gg (sequence number) into x[0..7], then release the slot
    auto take = [&](int gg, float2 (&x)[kGroupRows]) {
        const int gs = gg % kRingGroups;
        if (ok && !mbar_wait(&full[gs], (gg / kRingGroups) & 1)) {
            set_status(status, ST_ETIMEOUT);
            ok = false;
            g_fail = gg;
        }
#pragma unroll
        for (int i = 0; i < kGroupRows; ++i)
            x[i] = (ok && WCT_IDX_OK(status, gs * kGroupRows + i, kRingGroups * kGroupRows))
                       ? ring[gs * kGroupRows + i][tid]
                       : make_float2(0.f, 0.f);
        // after a timeout this thread releases no slot: a slot whose copy may still land is
        // never handed to the producer again (it then gives up on its own bounded wait)
        if (ok) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[gs])) : "memory");
    };
    for (int ph = 0; ph < n_phases; ++ph) {
        const int gbase = ph * n_groups;
        const float2 *Rp = Rt + (size_t)ph * r_phase_stride;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const float2 v = live ? Rp[(size_t)k * Fs + f] : make_float2(0.f, 0.f);
            rr[k] = make_float2(v.x, v.x);
            ri[k] = make_float2(v.y, v.y);
        }
        const bool acc = accumulate || ph > 0;
        float2 win[kWin];
        {
            // rows -4 .. 19: the upper half of group 0, groups 1 and 2
            float2 x[kGroupRows];
            take(gbase, x);
#pragma unroll
            for (int i = 0; i < 4; ++i) win[i] = x[4 + i];
            take(gbase + 1, x);
#pragma unroll
            for (int i = 0; i < kGroupRows; ++i) win[4 + i] = x[i];
            take(gbase + 2, x);
#pragma unroll
            for (int i = 0; i < kGroupRows; ++i) win[12 + i] = x[i];
        }
        float2 *dst = T + (size_t)w0 * Fs + f;
        for (int q = 0; q < n_blocks; ++q) {
            {
                float2 x[kGroupRows];
                take(gbase + q + kGroupLead, x);
#pragma unroll
                for (int i = 0; i < kGroupRows; ++i) win[2 * KC + i] = x[i];
            }
            const int nj = min(kOutBlock, n_out - kOutBlock * q);
#pragma unroll
            for (int j = 0; j < kOutBlock; ++j) {
                // packed pairs: A = sum x * (r.re, r.re), B = sum x * (r.im, r.im), so that
                // re = A.re - B.im and im = A.im + B.re (two FFMA2 per tap instead of four FFMA)
                float2 A = make_float2(0.f, 0.f), B = A, A2 = A, B2 = A;
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const float2 x = win[j + 2 * KC - k];
                    if (k & 1) {
                        A2 = fma2(x, rr[k], A2);
                        B2 = fma2(x, ri[k], B2);
                    } else {
                        A = fma2(x, rr[k], A);
                        B = fma2(x, ri[k], B);
                    }
                }
                A = add2(A, A2);
                B = add2(B, B2);
                if (live && j < nj &&
                    WCT_IDX_OK(status, (int64_t)(w0 + kOutBlock * q + j) * Fs + f, (int64_t)n_wires * Fs)) {
                    float2 v = make_float2(A.x - B.y, A.y + B.x);
                    if (n_phases > 1) {
                        float2 &t = tile[(kOutBlock * q + j) * kStageFB + tid];
                        const bool last = ph == n_phases - 1;
                        if (ph > 0) v = cadd(v, t);
                        if (!last) {
                            t = v;
                        } else {
                            if (accumulate) v = cadd(v, dst[(size_t)j * Fs]);
                            dst[(size_t)j * Fs] = v;
                        }
                    } else {
                        if (acc) v = cadd(v, dst[(size_t)j * Fs]);
                        dst[(size_t)j * Fs] = v;
                    }
                }
            }
            dst += (size_t)kOutBlock * Fs;
#pragma unroll
            for (int t = 0; t < 2 * KC; ++t) win[t] = win[t + kOutBlock];
        }
    }
    if (!ok && tid == 0) {
        // after a timeout: once the producer has stopped issuing (bounded), wait (bounded) for
        // every group it issued from the one that ran out on; they sit in distinct slots (a
        // slot is reissued only after this thread released it), so no copy lands in the
        // shared memory of a CTA that has left
        const long long t0 = clock64();
        while (!*(volatile int *)&s_prod_done && clock64() - t0 < kWaitCycles) {
        }
        const int issued = *(volatile int *)&s_issued;
        for (int g = g_fail; g < issued; ++g) mbar_wait(&full[g % kRingGroups], (g / kRingGroups) & 1);
    }
}

// Row activity of a library grid from the rasterizer's touched-tile flags (tiles of tile_w
// wires x the flag layout's ticks, n_tiles_t per band of wires): act_s[w] = 1 when some tile of
// wire w's band was touched (otherwise the row is all zero, and so is its spectrum), act_t[w] =
// 1 when some wire within +-KC of w is (otherwise the convolution's output row is zero).
// With n_phases > 1 (impact mode) the flags cover the phase grids stacked as one grid of
// n_phases * n_wires rows: act_s then has a byte per phase row and act_t[w] is set when some
// phase has a touched row within +-KC of w.
__global__ void k_row_activity(const uint32_t *__restrict__ flags, int n_tiles_t, int tile_w, int n_wires,
                               int n_phases, uint8_t *__restrict__ act_s, uint8_t *__restrict__ act_t) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    auto band = [&](int b) {
        const uint32_t *f = flags + (size_t)b * n_tiles_t;
        uint32_t any = 0;
        for (int t = 0; t < n_tiles_t; ++t) any |= f[t];
        return any != 0u;
    };
    if (r < n_phases * n_wires) act_s[r] = band(r / tile_w) ? 1 : 0;
    if (r < n_wires) {
        bool t_on = false;
        for (int ph = 0; ph < n_phases && !t_on; ++ph) {
            const int base = ph * n_wires;
            const int b0 = (base + max(r - KC, 0)) / tile_w, b1 = (base + min(r + KC, n_wires - 1)) / tile_w;
            for (int bb = b0; bb <= b1 && !t_on; ++bb) t_on = band(bb);
        }
        act_t[r] = t_on ? 1 : 0;
    }
}

// Twiddle tables on the device: tw[k] = exp(-2 pi i k / M) (k < M) and
// rtw[k] = exp(-2 pi i k / (2M)) (k <= M), evaluated in double precision.
__global__ void k_make_twiddles(float2 *__restrict__ tw, float2 *__restrict__ rtw, int M) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= M) {
        double sn, cs;
        sincospi(-(double)k / (double)M, &sn, &cs);          // angle -pi k / M
        rtw[k] = make_float2((float)cs, (float)sn);
        if (k < M) {
            sincospi(-2.0 * (double)k / (double)M, &sn, &cs);  // angle -2 pi k / M
            tw[k] = make_float2((float)cs, (float)sn);
        }
    }
}

// Self-test of the bounded wait: one thread waits on an mbarrier whose phase never completes
// (nothing arrives), gives up after `limit` cycles and records WCT_ETIMEOUT, as the library's
// kernels do when a copy never lands.
__global__ void k_wait_selftest(long long limit, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait(&bar, 0, limit)) set_status(status, ST_ETIMEOUT);
    }
}

__global__ void k_scale(float2 *__restrict__ a, int64_t n, float s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = cscale(a[i], s);
}

int pick_threads(int M) { return M >= 2048 ? 512 : (M >= 512 ? 256 : 128); }

}  // namespace

namespace {

int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

size_t device_smem_optin() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return (size_t)n;
}

size_t device_smem_per_sm() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    return (size_t)n;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// CTAs of k_wire_stage_tma resident on the whole current device (occupancy x SMs), computed
// once per device under a lock and cached.
constexpr int kMaxDevicesFft = 64;
std::mutex g_resident_mu;
int g_resident[kMaxDevicesFft] = {};

int wire_stage_resident() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesFft) {
        cudaGetLastError();
        return std::max(device_sms(), 1);
    }
    std::lock_guard<std::mutex> lock(g_resident_mu);
    if (g_resident[dev] == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wire_stage_tma, kStageFB + 32, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        g_resident[dev] = per_sm * std::max(device_sms(), 1);
    }
    return g_resident[dev];
}

// Row-transform schedule (FFTPlan::row_schedule): 0 = register-staged small CTAs (compiled
// lengths), 1 = persistent bulk-copy CTAs, one per SM, 2 = persistent paired CTAs, two per SM
// (compiled lengths; else 1), 3 = 2 with composite radices where compiled.
int row_kernel_choice(const FFTPlan &p) { return p.row_schedule; }

// The persistent bulk-copy kernels need 16-byte aligned rows (n_cols % 4 == 0, dense rows)
// and their five row-sized buffers in one CTA's shared memory.
bool use_row_tma(const FFTPlan &p, int64_t stride, int n_cols, const void *ptr) {
    return (n_cols % 4 == 0) && stride == n_cols && aligned16(ptr) && row_tma_smem_bytes(p.M) <= device_smem_optin() &&
           device_sms() > 0;
}

struct R2CKernels {
    template <class F>
    static auto get() { return k_row_r2c_tma<F>; }
};
struct C2RKernels {
    template <class F>
    static auto get() { return k_row_c2r_tma<F>; }
};

// Pick the compiled plan for the common lengths (M = 4900: 9600 ticks, M = 3125: 6000 ticks,
// M = 625: 1024 ticks), else the runtime-radix kernel; set its shared-memory limit; launch.
template <class Launch, class K>
cudaError_t launch_row_tma_kernel(const FFTPlan &p, size_t smem, int grid, cudaStream_t s, Launch &&launch, K) {
    (void)grid;
    (void)s;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        launch(kern);
        return cudaGetLastError();
    };
    auto is = [&](std::initializer_list<int> rs) {
        if ((int)rs.size() != p.n_stages) return false;
        int k = 0;
        for (int r : rs)
            if (p.radix[k++] != r) return false;
        return true;
    };
    if (is({7, 4, 5, 5, 7})) return go(K::template get<CompiledFft<CtPlan<7, 4, 5, 5, 7>>>());
    if (is({5, 5, 5, 5, 5})) return go(K::template get<CompiledFft<CtPlan<5, 5, 5, 5, 5>>>());
    if (is({5, 5, 5, 5})) return go(K::template get<CompiledFft<CtPlan<5, 5, 5, 5>>>());
    return go(K::template get<RuntimeFft>());
}

// Register-staged kernels for the compiled lengths (4900, 3125, 625); false if none applies.
template <bool R2C, class Launch>
bool launch_row_rs(const FFTPlan &p, Launch &&launch, cudaError_t &err) {
    auto is = [&](std::initializer_list<int> rs) {
        if ((int)rs.size() != p.n_stages) return false;
        int k = 0;
        for (int r : rs)
            if (p.radix[k++] != r) return false;
        return true;
    };
    const size_t smem = sizeof(float2) * (size_t)p.M;
    auto go = [&](auto kern) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) {
            launch(kern, smem);
            err = cudaGetLastError();
        }
        return true;
    };
    if constexpr (R2C) {
        if (is({7, 4, 5, 5, 7})) return go(k_row_r2c_rs<CtPlan<7, 4, 5, 5, 7>>);
        if (is({5, 5, 5, 5, 5})) return go(k_row_r2c_rs<CtPlan<5, 5, 5, 5, 5>>);
        if (is({5, 5, 5, 5})) return go(k_row_r2c_rs<CtPlan<5, 5, 5, 5>>);
    } else {
        if (is({7, 4, 5, 5, 7})) return go(k_row_c2r_rs<CtPlan<7, 4, 5, 5, 7>>);
        if (is({5, 5, 5, 5, 5})) return go(k_row_c2r_rs<CtPlan<5, 5, 5, 5, 5>>);
        if (is({5, 5, 5, 5})) return go(k_row_c2r_rs<CtPlan<5, 5, 5, 5>>);
    }
    return false;
}

// Paired kernels for the compiled lengths (4900, 3125, 625); false if none applies.  With
// `composite`, M = 4900 runs three Stockham passes of radices 25, 28, 7 and M = 3125 three of
// 5, 25, 25 (composite butterflies, 256 threads of up to 128 registers) instead of five passes
// of 7, 4, 5, 5, 7 or 5, 5, 5, 5, 5 (512 threads): 40 % fewer shared-memory wavefronts under
// the bank model of the plan's stage ordering (at 3456 x 9600: forward 72 -> 68 us, inverse
// 83 -> 78 us; the rest is copy latency and barriers, not shared-memory bandwidth).
template <bool R2C, class Launch>
bool launch_row_pair(const FFTPlan &p, bool composite, Launch &&launch, cudaError_t &err) {
    auto is = [&](std::initializer_list<int> rs) {
        if ((int)rs.size() != p.n_stages) return false;
        int k = 0;
        for (int r : rs)
            if (p.radix[k++] != r) return false;
        return true;
    };
    const size_t smem = row_pair_smem_bytes(p.M);
    if (2 * smem + 2048 > (size_t)device_smem_per_sm() || smem > (size_t)device_smem_optin()) return false;
    auto go = [&](auto kern, int threads) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) {
            launch(kern, smem, threads);
            err = cudaGetLastError();
        }
        return true;
    };
    constexpr int T = kPairThreads, TC = kPairThreadsComposite;
    if constexpr (R2C) {
        if (composite && is({7, 4, 5, 5, 7})) return go(k_row_r2c_pair<TC, 25, 28, 7>, TC);
        if (composite && is({5, 5, 5, 5, 5})) return go(k_row_r2c_pair<TC, 5, 25, 25>, TC);
        if (is({7, 4, 5, 5, 7})) return go(k_row_r2c_pair<T, 7, 4, 5, 5, 7>, T);
        if (is({5, 5, 5, 5, 5})) return go(k_row_r2c_pair<T, 5, 5, 5, 5, 5>, T);
        if (is({5, 5, 5, 5})) return go(k_row_r2c_pair<T, 5, 5, 5, 5>, T);
    } else {
        if (composite && is({7, 4, 5, 5, 7})) return go(k_row_c2r_pair<TC, 25, 28, 7>, TC);
        if (composite && is({5, 5, 5, 5, 5})) return go(k_row_c2r_pair<TC, 5, 25, 25>, TC);
        if (is({7, 4, 5, 5, 7})) return go(k_row_c2r_pair<T, 7, 4, 5, 5, 7>, T);
        if (is({5, 5, 5, 5, 5})) return go(k_row_c2r_pair<T, 5, 5, 5, 5, 5>, T);
        if (is({5, 5, 5, 5})) return go(k_row_c2r_pair<T, 5, 5, 5, 5>, T);
    }
    return false;
}

}  // namespace

cudaError_t launch_row_r2c(const FFTPlan &p, const float *in, int64_t in_stride, int n_in_cols, int n_rows,
                           float2 *spec, cudaStream_t s, int32_t *status, const uint8_t *act) {
    if (n_rows <= 0) return cudaSuccess;
    if (row_kernel_choice(p) == 0 && (n_in_cols % 4 == 0) && in_stride == n_in_cols && aligned16(in) && aligned16(spec)) {
        cudaError_t err = cudaSuccess;
        if (launch_row_rs<true>(p, [&](auto kern, size_t smem) {
                kern<<<n_rows, kRsThreads, smem, s>>>(p, in, n_in_cols, spec);
            }, err))
            return err;
    }
    if (row_kernel_choice(p) >= 2 && use_row_tma(p, in_stride, n_in_cols, in) && aligned16(spec) && 2 * p.M >= n_in_cols) {
        cudaError_t err = cudaSuccess;
        const int grid = std::min(n_rows, 2 * device_sms());
        if (launch_row_pair<true>(p, row_kernel_choice(p) == 3, [&](auto kern, size_t smem, int threads) {
                kern<<<grid, threads, smem, s>>>(p, in, n_rows, n_in_cols, spec, status, act);
            }, err))
            return err;
    }
    if (use_row_tma(p, in_stride, n_in_cols, in) && aligned16(spec)) {
        const size_t smem = row_tma_smem_bytes(p.M);
        const int grid = std::min(n_rows, device_sms());
        return launch_row_tma_kernel(p, smem, grid, s, [&](auto kern) {
            kern<<<grid, kRowThreads, smem, s>>>(p, in, n_rows, n_in_cols, spec, status);
        }, R2CKernels{});
    }
    const int T = pick_threads(p.M);
    const size_t smem = 2 * sizeof(float2) * (size_t)p.M;
    cudaError_t e = cudaFuncSetAttribute(k_row_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_row_r2c<<<n_rows, T, smem, s>>>(p, in, in_stride, n_in_cols, spec);
    return cudaGetLastError();
}

cudaError_t launch_row_c2r(const FFTPlan &p, const float2 *spec, int n_rows, float *out, int64_t out_stride,
                           int n_out_cols, cudaStream_t s, int32_t *status, const uint8_t *act) {
    if (n_rows <= 0) return cudaSuccess;
    if (row_kernel_choice(p) == 0 && (n_out_cols % 4 == 0) && out_stride == n_out_cols && aligned16(out) &&
        aligned16(spec)) {
        cudaError_t err = cudaSuccess;
        if (launch_row_rs<false>(p, [&](auto kern, size_t smem) {
                kern<<<n_rows, kRsThreads, smem, s>>>(p, spec, out, n_out_cols);
            }, err))
            return err;
    }
    if (row_kernel_choice(p) >= 2 && use_row_tma(p, out_stride, n_out_cols, out) && aligned16(spec) &&
        2 * p.M >= n_out_cols) {
        cudaError_t err = cudaSuccess;
        const int grid = std::min(n_rows, 2 * device_sms());
        if (launch_row_pair<false>(p, row_kernel_choice(p) == 3, [&](auto kern, size_t smem, int threads) {
                kern<<<grid, threads, smem, s>>>(p, spec, n_rows, out, n_out_cols, status, act);
            }, err))
            return err;
    }
    if (use_row_tma(p, out_stride, n_out_cols, out) && aligned16(spec)) {
        const size_t smem = row_tma_smem_bytes(p.M);
        const int grid = std::min(n_rows, device_sms());
        return launch_row_tma_kernel(p, smem, grid, s, [&](auto kern) {
            kern<<<grid, kRowThreads, smem, s>>>(p, spec, n_rows, out, n_out_cols, status);
        }, C2RKernels{});
    }
    const int T = pick_threads(p.M);
    const size_t smem = 2 * sizeof(float2) * (size_t)p.M;
    cudaError_t e = cudaFuncSetAttribute(k_row_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_row_c2r<<<n_rows, T, smem, s>>>(p, spec, out, out_stride, n_out_cols);
    return cudaGetLastError();
}

cudaError_t launch_wire_stage(const FFTPlan &p, const float2 *spec, const float2 *resp_spec, int n_wires, float2 *out,
                              cudaStream_t s, int32_t *status, const ClearJob *clear, bool accumulate, int n_phases,
                              const uint8_t *act) {
    if (n_wires <= 0) return cudaSuccess;
    const ClearJob job = clear ? *clear : ClearJob{};
    if (aligned16(spec) && (p.Fs % 2) == 0 && (p.Fu % 2) == 0) {
        // Output wires per CTA: a CTA's time grows with the rows it streams (wpc + 20 halo),
        // and the launch takes ceil(CTAs / resident CTAs) waves, so pick the wpc that
        // minimises waves x (wpc + 20): a last, nearly empty wave costs a full CTA time.
        const int fb = (p.Fu + kStageFB - 1) / kStageFB;
        // impact mode: the phases' sum of a CTA's outputs lives in shared memory, so runs are
        // short (at most kImpactWires output wires)
        const int max_c = n_phases > 1 ? kImpactWires : kStageWiresMax;
        const size_t dyn = n_phases > 1 ? sizeof(float2) * (size_t)kImpactWires * kStageFB : 0;
        int resident = 0;
        if (n_phases > 1) {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wire_stage_tma, kStageFB + 32, dyn) != cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            resident = per_sm * std::max(device_sms(), 1);
        } else {
            resident = wire_stage_resident();
        }
        int wpc = max_c;
        int64_t best = INT64_MAX;
        for (int c = 16; c <= max_c; ++c) {
            const int64_t ctas = (int64_t)fb * ((n_wires + c - 1) / c);
            const int64_t cost = (ctas + resident - 1) / resident * (c + 2 * KC);
            if (cost < best) {
                best = cost;
                wpc = c;
            }
        }
        dim3 grid(fb, (n_wires + wpc - 1) / wpc);
        if (dyn) {
            const cudaError_t e = cudaFuncSetAttribute(k_wire_stage_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
        }
        k_wire_stage_tma<<<grid, kStageFB + 32, dyn, s>>>(spec, resp_spec, p.Fs, p.Fu, n_wires, wpc, out, status, job,
                                                        accumulate ? 1 : 0, n_phases, (int64_t)n_wires * p.Fs,
                                                        (int64_t)KW * p.Fs, act);
        return cudaGetLastError();
    }
    if (n_phases > 1) {
        // fallback kernel: one phase per launch, accumulating
        for (int ph = 0; ph < n_phases; ++ph) {
            const cudaError_t e = launch_wire_stage(p, spec + (size_t)ph * n_wires * p.Fs,
                                                    resp_spec + (size_t)ph * KW * p.Fs, n_wires, out, s, status,
                                                    ph == 0 ? clear : nullptr, accumulate || ph > 0, 1);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    dim3 grid((p.Fu + kStageThreads - 1) / kStageThreads, (n_wires + kStageRun - 1) / kStageRun);
    k_wire_stage<<<grid, kStageThreads, 0, s>>>(spec, resp_spec, p.Fs, p.Fu, n_wires, out, accumulate ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && job.grid) {
        k_clear_tiles_fft<<<job.n_tiles < 2 * 152 ? job.n_tiles : 2 * 152, 256, 0, s>>>(job);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_row_activity(const uint32_t *flags, int n_tiles_t, int tile_w, int n_wires, uint8_t *act_s,
                                uint8_t *act_t, cudaStream_t s, int n_phases) {
    const int rows = n_phases * n_wires;
    if (rows <= 0) return cudaSuccess;
    k_row_activity<<<(rows + 255) / 256, 256, 0, s>>>(flags, n_tiles_t, tile_w, n_wires, n_phases, act_s, act_t);
    return cudaGetLastError();
}

cudaError_t launch_make_twiddles(const FFTPlan &p, cudaStream_t s) {
    k_make_twiddles<<<(p.M + 256) / 256, 256, 0, s>>>(p.tw, p.rtw, p.M);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long limit, int32_t *status, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(limit, status);
    return cudaGetLastError();
}

cudaError_t launch_scale_spectrum(float2 *spec, int64_t n, float scale, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(spec, n, scale);
    return cudaGetLastError();
}

}  // namespace wct
