// Shared device helpers of the PD-R CUDA library: complex arithmetic on
// float2/double2, the Kaiser-Bessel weight, Philox-4x64-10 and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdgb {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename R> using cplx_t = typename CplxOf<R>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C{}.x) re, decltype(C{}.x) im) {
    C c; c.x = re; c.y = im; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (sign < 0) or +i (sign > 0)
template <int SIGN, typename C> __device__ __forceinline__ C mul_i(C a) {
    return SIGN < 0 ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
}

__device__ __forceinline__ float bessel_i0(float z) { return cyl_bessel_i0f(z); }
__device__ __forceinline__ double bessel_i0(double z) { return cyl_bessel_i0(z); }

// Kaiser-Bessel weight I0(beta sqrt(1 - (2t/J)^2)) for |t| <= J/2, else 0.
template <typename R> __device__ __forceinline__ R kb_weight(R t, R two_over_j, R beta) {
    R q = t * two_over_j;
    R arg = R(1) - q * q;
    return arg >= R(0) ? bessel_i0(beta * sqrt(arg)) : R(0);
}

// Philox-4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11); returns word 0.
__host__ __device__ inline uint64_t philox_word0(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
#else
        unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
    return c0;
}
// u in [0, 1) from the top 53 bits of word 0.
__host__ __device__ inline double philox_uniform(uint64_t seed, uint64_t t, uint64_t stream, uint64_t index) {
    return (double)(philox_word0(t, stream, index, 0, seed, 0) >> 11) * (1.0 / 9007199254740992.0);
}

// Deterministic block-wide sum of a double for any blockDim.x that is a multiple
// of 32 (fixed shuffle tree per warp, then warp 0). sh must hold 32 doubles.
// The result is valid in thread 0.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// dst[i] = load(i) for i < n over the CTA, with U independent global loads in flight per
// thread: the plain strided loop waits for each load before issuing the next, which
// leaves small grids bound by one memory latency per element a thread stages.
template <int U, typename T, class F>
__device__ __forceinline__ void stage_batched(T* dst, int n, const F& load) {
    for (int base = threadIdx.x; base < n; base += U * (int)blockDim.x) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * (int)blockDim.x;
            if (i < n) v[u] = load(i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * (int)blockDim.x;
            if (i < n) dst[i] = v[u];
        }
    }
}

// Allow a kernel `bytes` of dynamic shared memory. Static plus dynamic shared memory
// above 48 KB needs the opt-in attribute, so it is always set to the requested size.
template <typename K> inline cudaError_t ensure_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace pdgb
