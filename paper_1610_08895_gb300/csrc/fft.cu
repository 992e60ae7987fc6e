// Oversampled 2-D FFT passes of Phi = G F Z and of its adjoint (Sec. 2), as
// shared-memory Stockham transforms of compile-time length.
//
// The grid is (2 ny) x (2 nx) but only ny x nx of its input cells are non-zero
// (zero padding by Z), and the adjoint only needs ny x nx of its outputs (the
// crop of Z^T). Every pass therefore runs half-length transforms: with a length
// 2n transform split into even and odd outputs (forward) or inputs (inverse),
//   X[2j + r] = sum_l (x_l W_2n^{r l}) W_n^{j l},
//   x_l       = E_l + W_2n^{-l} O_l,  E/O = inverse length-n transforms of even/odd inputs.
// The image is real, so F Z x is Hermitian, B[-k] = conj(B[k]): the forward passes
// produce only the columns kx = 0 .. nx (the "half grid"), transforming two image rows
// at once as the real and imaginary parts of one complex row. The adjoint needs only
// Re(Z^T F^H U) = Z^T F^H H with H the Hermitian part (U[k] + conj(U[-k])) / 2, whose
// column transforms are again Hermitian in kx: the inverse column pass transforms the
// columns kx = 0 .. nx of H and the inverse row pass two rows at once.
// Layouts: images are row-major [ny][nx]; the half-grid intermediates (t1) and the
// forward output use column panels [nx/4 + 1][rows][4]; the gridded U is the full
// panel grid [Kx/4][Ky][4].
#include "common.cuh"
#include "plan.hpp"

namespace pdgb {

// o * exp(SIGN * 2 pi i j / 16) for j in [0, 8)
template <int SIGN, typename C> __device__ __forceinline__ C rot16(C o, int j) {
    using R = decltype(o.x);
    const R S1 = R(0.38268343236508977172845998403039886676134456248563);
    const R C1 = R(0.92387953251128675612818318939678828682241662586364);
    const R H = R(0.70710678118654752440084436210484903928483593768847);
    switch (j) {
        case 0: return o;
        case 1: return cmul(o, mk<C>(C1, SIGN * S1));
        case 2: return mk<C>(H * (o.x - SIGN * o.y), H * (o.y + SIGN * o.x));
        case 3: return cmul(o, mk<C>(S1, SIGN * C1));
        case 4: return mul_i<SIGN>(o);
        case 5: return cmul(o, mk<C>(-S1, SIGN * C1));
        case 6: return mk<C>(-H * (o.x + SIGN * o.y), H * (SIGN * o.x - o.y));
        default: return cmul(o, mk<C>(-C1, SIGN * S1));
    }
}

// In-register DFT of size RAD (power of two <= 16), in place, by radix-2
// decimation in frequency: each pass combines a = v[i], b = v[i + h] into
// v[i] = a + b and v[i + h] = (a - b) exp(SIGN 2 pi i j / 2h). The result is in
// bit-reversed order: X[k] = v[bitrev(k)].
template <int RAD, int SIGN, typename C> __device__ __forceinline__ void dft_dif(C* v) {
#pragma unroll
    for (int h = RAD / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int base = 0; base < RAD; base += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C a = v[base + j], b = v[base + j + h];
                v[base + j] = cadd(a, b);
                v[base + j + h] = rot16<SIGN>(csub(a, b), j * (8 / h));
            }
        }
    }
}

template <int RAD> __host__ __device__ constexpr int bitrev(int k) {
    int r = 0;
    for (int m = RAD >> 1, q = 1; m >= 1; m >>= 1, q <<= 1)
        if (k & m) r |= q;
    return r;
}

// Compile-time shape of the length-N transforms of one precision: each thread holds EPT
// elements per stage (radix EPT stages after a first stage of the remaining radix), and
// sequences are stored with one pad element per PADV elements against bank conflicts.
template <typename R, int N> struct Shape {
    static constexpr int RAD = sizeof(R) == 4 ? 16 : 8;
    static constexpr int EPT = N < RAD ? N : RAD;
    static constexpr int PADV = sizeof(R) == 4 ? 16 : 8;
    static constexpr int PN = N + N / PADV;            // padded sequence length
    static constexpr int first_radix() {
        int r = N;
        while (r > EPT) r /= EPT;
        return r;
    }
};
template <typename R> __device__ __forceinline__ int padi(int l) { return l + (l >> (sizeof(R) == 4 ? 4 : 3)); }

// One Stockham autosort stage of radix RADS over NSEQ sequences of length N held in
// shared memory (sequence c at s + c * PN, padded). NS is the product of the radices of
// the earlier stages. Butterfly i (k = i mod NS) takes x[i + r N/RADS], multiplies by
// W^{k r / (NS RADS)} (from twK[m] = exp(-2 pi i m / (2N)), conjugated for SIGN > 0),
// transforms, and stores X_r at (i / NS) NS RADS + k + r NS. All reads happen before the
// barrier, all writes after it, so the stage works in place.
template <typename R, int N, int RADS, int NS, int SIGN, int NSEQ>
__device__ __forceinline__ void stage(cplx_t<R>* s, const cplx_t<R>* __restrict__ twK) {
    using C2 = cplx_t<R>;
    using S = Shape<R, N>;
    constexpr int NJ = N / RADS, JOBS = S::EPT / RADS, NT = N * NSEQ / S::EPT;
    const bool act = NT >= 32 || (int)threadIdx.x < NT;     // CTAs are at least one warp
    C2 v[JOBS][RADS];
#pragma unroll
    for (int jb = 0; jb < JOBS; ++jb) {
        const int job = act ? threadIdx.x + jb * NT : 0;
        const int c = job / NJ, i = job % NJ, k = i % NS;
        const C2* src = s + c * S::PN;
#pragma unroll
        for (int r = 0; r < RADS; ++r) {
            C2 a = src[padi<R>(i + r * NJ)];
            if (NS > 1 && r > 0) {
                C2 w = __ldg(&twK[k * r * (2 * N / (NS * RADS))]);
                if (SIGN > 0) w.y = -w.y;
                a = cmul(a, w);
            }
            v[jb][r] = a;
        }
        dft_dif<RADS, SIGN>(v[jb]);
    }
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < JOBS; ++jb) {
        if (!act) break;
        const int job = threadIdx.x + jb * NT;
        const int c = job / NJ, i = job % NJ, k = i % NS;
        C2* dst = s + c * S::PN;
        const int base = (i / NS) * NS * RADS + k;
#pragma unroll
        for (int r = 0; r < RADS; ++r) dst[padi<R>(base + r * NS)] = v[jb][bitrev<RADS>(r)];
    }
    __syncthreads();
}

template <typename R, int N, int NS, int SIGN, int NSEQ>
__device__ __forceinline__ void stages(cplx_t<R>* s, const cplx_t<R>* __restrict__ twK) {
    if constexpr (NS < N) {
        constexpr int RADS = NS == 1 ? Shape<R, N>::first_radix() : Shape<R, N>::EPT;
        stage<R, N, RADS, NS, SIGN, NSEQ>(s, twK);
        stages<R, N, NS * RADS, SIGN, NSEQ>(s, twK);
    }
}

// NSEQ unnormalised length-N DFTs (SIGN -1 forward, +1 inverse) of the sequences in s,
// natural order in and out. Every thread of the CTA (N NSEQ / EPT of them) takes part.
template <typename R, int N, int SIGN, int NSEQ>
__device__ __forceinline__ void fft_smem(cplx_t<R>* s, const cplx_t<R>* __restrict__ twK) {
    stages<R, N, 1, SIGN, NSEQ>(s, twK);
}

// e = threadIdx.x, threadIdx.x + NT, ... < total, with the global loads of UB consecutive
// steps issued before any of their shared-memory stores (a plain strided loop waits for
// each load in turn, which leaves these passes bound by one memory latency per step).
template <int UB, int NT, class Ld, class St>
__device__ __forceinline__ void batched_loop(int total, const Ld& ld, const St& st) {
    using V = decltype(ld(0));
    for (int base = threadIdx.x; base < total; base += UB * NT) {
        V v[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = base + u * NT;
            if (e < total) v[u] = ld(e);
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = base + u * NT;
            if (e < total) st(e, v[u]);
        }
    }
}

// Rows (pairs) per CTA of the row passes and columns per CTA of the column passes:
// as many as keep a CTA at 512 threads (so a thread may hold 128 registers), at most 4,
// at least 1 (the longest transforms then take 1024 threads).
template <typename R, int N> struct PassShape {
    static constexpr int EPT = Shape<R, N>::EPT;
    static constexpr int FIT = 512 * EPT / (2 * N);
    static constexpr int PAIRS = FIT < 1 ? 1 : (FIT > 4 ? 4 : FIT);
    static constexpr int CQ = PAIRS;
    static constexpr int NT_ROWS = 2 * PAIRS * N / EPT < 32 ? 32 : 2 * PAIRS * N / EPT;
    static constexpr int NT_COLS = 2 * CQ * N / EPT < 32 ? 32 : 2 * CQ * N / EPT;
    static constexpr size_t SMEM_ROWS = (size_t)2 * PAIRS * Shape<R, N>::PN * sizeof(cplx_t<R>);
    static constexpr size_t SMEM_COLS = (size_t)2 * CQ * Shape<R, N>::PN * sizeof(cplx_t<R>);
    // two CTAs per SM where the threads allow it (the register budget per thread follows)
    static constexpr int MIN_CTAS_ROWS = NT_ROWS <= 512 ? 2 : 1;
    static constexpr int MIN_CTAS_COLS = NT_COLS <= 512 ? 2 : 1;
};

// ---------------------------------------------------------------------------
// Forward row pass (Z, then F along x) of two image rows a = iy0 + 2 pr, b = a + 1 per
// pair: z = Z x_a + i Z x_b. Sequence 2 pr holds z for the even outputs, 2 pr + 1 the
// pre-twiddled z for the odd ones. Output: the half spectrum kx = 0 .. nx of each row,
// X_a[k] = (Z[k] + conj Z[-k]) / 2 and X_b[k] = (Z[k] - conj Z[-k]) / (2i), into t1.
template <typename R, int N>
__global__ void __launch_bounds__(PassShape<R, N>::NT_ROWS, PassShape<R, N>::MIN_CTAS_ROWS) k_fwd_rows(
    const R* __restrict__ x, cplx_t<R>* __restrict__ t1, const R* __restrict__ cx, const R* __restrict__ cy,
    const cplx_t<R>* __restrict__ twx, int ny, int64_t t1_stride) {
    using C2 = cplx_t<R>;
    using S = Shape<R, N>;
    using P = PassShape<R, N>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    x += (int64_t)blockIdx.y * ny * N;                 // image blockIdx.y of a batch
    t1 += (int64_t)blockIdx.y * t1_stride;
    constexpr int NT = P::NT_ROWS, Kx = 2 * N;
    const int iy0 = blockIdx.x * 2 * P::PAIRS;
    struct In { R va, vb; C2 w; };
    batched_loop<4, NT>(P::PAIRS * N, [&](int e) {
        const int pr = e / N, ix = e % N;
        const int a = iy0 + 2 * pr;
        const R c = cx[ix];
        const int lc = ix - N / 2;
        return In{x[(int64_t)a * N + ix] * c * cy[a], x[(int64_t)(a + 1) * N + ix] * c * cy[a + 1],
                  __ldg(&twx[lc & (Kx - 1)])};
    }, [&](int e, const In& v) {
        const int pr = e / N, ix = e % N;
        const int m = padi<R>((ix - N / 2) & (N - 1));
        s[(2 * pr) * S::PN + m] = mk<C2>(v.va, v.vb);
        s[(2 * pr + 1) * S::PN + m] = mk<C2>(v.va * v.w.x - v.vb * v.w.y, v.va * v.w.y + v.vb * v.w.x);
    });
    __syncthreads();
    fft_smem<R, N, -1, 2 * P::PAIRS>(s, twx);
    // outputs ordered (panel, row, slot): 2 PAIRS rows x 4 slots of a panel are contiguous
    constexpr int NPH = N / 4 + 1;
    for (int e = threadIdx.x; e < NPH * 2 * P::PAIRS * 4; e += NT) {
        const int q = e & 3, rr = (e >> 2) % (2 * P::PAIRS), pp = (e >> 2) / (2 * P::PAIRS);
        const int kx = 4 * pp + q;
        if (kx > N) continue;
        const int pr = rr >> 1;
        const C2* ev = s + (2 * pr) * S::PN;
        const C2* od = ev + S::PN;
        C2 z, zm;
        if ((kx & 1) == 0) {
            const int j = kx >> 1;
            z = ev[padi<R>(j & (N - 1))];
            zm = ev[padi<R>((N - j) & (N - 1))];
        } else {
            const int j = kx >> 1;
            z = od[padi<R>(j)];
            zm = od[padi<R>(N - 1 - j)];
        }
        const C2 out = (rr & 1) ? mk<C2>(R(0.5) * (z.y + zm.y), R(0.5) * (zm.x - z.x))
                                : mk<C2>(R(0.5) * (z.x + zm.x), R(0.5) * (z.y - zm.y));
        t1[((int64_t)pp * ny + iy0 + rr) * 4 + q] = out;
    }
}

// Forward column pass (F along y) of CQ half-grid columns of one panel: sequence qq holds
// column q0 + qq for the even outputs, CQ + qq the pre-twiddled column for the odd ones.
template <typename R, int N>
__global__ void __launch_bounds__(PassShape<R, N>::NT_COLS, PassShape<R, N>::MIN_CTAS_COLS) k_fwd_cols(
    const cplx_t<R>* __restrict__ t1, cplx_t<R>* __restrict__ gb, const cplx_t<R>* __restrict__ twy,
    int64_t t1_stride, int64_t gb_stride) {
    using C2 = cplx_t<R>;
    using S = Shape<R, N>;
    using P = PassShape<R, N>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    t1 += (int64_t)blockIdx.y * t1_stride;
    gb += (int64_t)blockIdx.y * gb_stride;
    constexpr int NT = P::NT_COLS, CQ = P::CQ, Ky = 2 * N, PER = 4 / CQ;
    const int p = blockIdx.x / PER, q0 = (blockIdx.x % PER) * CQ;
    const C2* src = t1 + (int64_t)p * N * 4 + q0;
    struct In { C2 val, w; };
    batched_loop<8, NT>(N * CQ, [&](int e) {
        const int iy = e / CQ, qq = e % CQ;
        return In{src[iy * 4 + qq], __ldg(&twy[(iy - N / 2) & (Ky - 1)])};
    }, [&](int e, const In& v) {
        const int iy = e / CQ, qq = e % CQ;
        const int m = padi<R>((iy - N / 2) & (N - 1));
        s[qq * S::PN + m] = v.val;
        s[(CQ + qq) * S::PN + m] = cmul(v.val, v.w);
    });
    __syncthreads();
    fft_smem<R, N, -1, 2 * CQ>(s, twy);
    C2* dst = gb + (int64_t)p * Ky * 4 + q0;
    for (int e = threadIdx.x; e < Ky * CQ; e += NT) {
        const int ky = e / CQ, qq = e % CQ;
        dst[ky * 4 + qq] = s[((ky & 1) * CQ + qq) * S::PN + padi<R>(ky >> 1)];
    }
}

// Inverse column pass (F^H along y, crop to ny rows) of the Hermitian part of U for the
// half-grid columns kx = 4 p + q0 + qq: h[ky] = (U[ky][kx] + conj U[-ky][-kx]) / 2, its
// even inputs in sequence qq and odd inputs in CQ + qq; the cropped row iy is
// E[m] + conj(W_2ny^lc) O[m] with lc = iy - ny/2, m = lc mod ny.
template <typename R, int N>
__global__ void __launch_bounds__(PassShape<R, N>::NT_COLS, PassShape<R, N>::MIN_CTAS_COLS) k_inv_cols(
    const cplx_t<R>* __restrict__ U, cplx_t<R>* __restrict__ t1, const cplx_t<R>* __restrict__ twy, int Kx,
    int64_t t1_stride) {
    using C2 = cplx_t<R>;
    using S = Shape<R, N>;
    using P = PassShape<R, N>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    U += (int64_t)blockIdx.y * Kx * 2 * N;
    t1 += (int64_t)blockIdx.y * t1_stride;
    constexpr int NT = P::NT_COLS, CQ = P::CQ, Ky = 2 * N, PER = 4 / CQ;
    const int p = blockIdx.x / PER, q0 = (blockIdx.x % PER) * CQ;
    struct In { C2 u, um; };
    batched_loop<8, NT>(Ky * CQ, [&](int e) {
        const int ky = e / CQ, qq = e % CQ;
        const int kx = 4 * p + q0 + qq;
        const int mkx = (Kx - kx) & (Kx - 1), mky = (Ky - ky) & (Ky - 1);
        return In{U[panel_off(ky, kx, Ky)], U[panel_off(mky, mkx, Ky)]};
    }, [&](int e, const In& v) {
        const int ky = e / CQ, qq = e % CQ;
        s[((ky & 1) * CQ + qq) * S::PN + padi<R>(ky >> 1)] =
            mk<C2>(R(0.5) * (v.u.x + v.um.x), R(0.5) * (v.u.y - v.um.y));
    });
    __syncthreads();
    fft_smem<R, N, +1, 2 * CQ>(s, twy);
    C2* dst = t1 + (int64_t)p * N * 4 + q0;
    for (int e = threadIdx.x; e < N * CQ; e += NT) {
        const int iy = e / CQ, qq = e % CQ;
        const int lc = iy - N / 2;
        const int m = padi<R>(lc & (N - 1));
        const C2 w = cconj(__ldg(&twy[lc & (Ky - 1)]));
        dst[iy * 4 + qq] = cadd(s[qq * S::PN + m], cmul(w, s[(CQ + qq) * S::PN + m]));
    }
}

// Inverse row pass (F^H along x of the Hermitian rows, crop, deapodise) of two rows at
// once: Z[k] = T_a[k] + i T_b[k] with T[2nx - k] = conj T[k], so F^H Z = out_a + i out_b.
// Mode 0 stores Re(Phi^H)-type output; mode 1 runs the primal update of Alg. 1 steps
// 17-18 as epilogue with per-CTA FP64 partial norms.
template <typename R, int N>
__global__ void __launch_bounds__(PassShape<R, N>::NT_ROWS, PassShape<R, N>::MIN_CTAS_ROWS) k_inv_rows(
    const cplx_t<R>* __restrict__ t1, R* __restrict__ out, const R* __restrict__ cx, const R* __restrict__ cy,
    const cplx_t<R>* __restrict__ twx, int ny, int mode, R tau, R sigma, R varsigma, R* __restrict__ xs,
    R* __restrict__ xt, const R* __restrict__ st_, double* __restrict__ part, int64_t t1_stride) {
    using C2 = cplx_t<R>;
    using S = Shape<R, N>;
    using P = PassShape<R, N>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    C2* s = reinterpret_cast<C2*>(smraw);
    t1 += (int64_t)blockIdx.y * t1_stride;             // image blockIdx.y of a batch (mode 0)
    if (mode == 0) out += (int64_t)blockIdx.y * ny * N;
    constexpr int NT = P::NT_ROWS, Kx = 2 * N, NPH = N / 4 + 1;
    const int iy0 = blockIdx.x * 2 * P::PAIRS;
    struct In { C2 ta, tb; };
    batched_loop<8, NT>(NPH * P::PAIRS * 4, [&](int e) {
        const int q = e & 3, pr = (e >> 2) % P::PAIRS, pp = (e >> 2) / P::PAIRS;
        const int a = iy0 + 2 * pr;
        In v;
        if (4 * pp + q <= N) { v.ta = t1[((int64_t)pp * ny + a) * 4 + q]; v.tb = t1[((int64_t)pp * ny + a + 1) * 4 + q]; }
        return v;
    }, [&](int e, const In& v) {
        const int q = e & 3, pr = (e >> 2) % P::PAIRS, pp = (e >> 2) / P::PAIRS;
        const int k = 4 * pp + q;
        if (k > N) return;
        C2* seq = s + (2 * pr + (k & 1)) * S::PN;
        seq[padi<R>(k >> 1)] = mk<C2>(v.ta.x - v.tb.y, v.ta.y + v.tb.x);
        if (k != 0 && k != N) seq[padi<R>((Kx - k) >> 1)] = mk<C2>(v.ta.x + v.tb.y, v.tb.x - v.ta.y);
    });
    __syncthreads();
    fft_smem<R, N, +1, 2 * P::PAIRS>(s, twx);
    R adx = R(0), ax = R(0);
    for (int e = threadIdx.x; e < P::PAIRS * N; e += NT) {
        const int pr = e / N, ix = e % N;
        const int lc = ix - N / 2;
        const int m = padi<R>(lc & (N - 1));
        const C2 w = cconj(__ldg(&twx[lc & (Kx - 1)]));
        const C2* ev = s + (2 * pr) * S::PN;
        const C2 z = cadd(ev[m], cmul(w, ev[S::PN + m]));
        const R c = cx[ix];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int iy = iy0 + 2 * pr + h;
            const R g = (h ? z.y : z.x) * c * cy[iy];
            const int64_t idx = (int64_t)iy * N + ix;
            if (mode == 0) {
                out[idx] = g;
            } else {
                const R xo = xs[idx];
                R xn = xo - tau * (sigma * st_[idx] + varsigma * g);
                xn = xn > R(0) ? xn : R(0);
                xt[idx] = R(2) * xn - xo;
                xs[idx] = xn;
                const R dd = xn - xo;
                adx += dd * dd;
                ax += xn * xn;
            }
        }
    }
    if (mode == 1) {
        const double sdx = block_sum((double)adx, red);
        const double sx = block_sum((double)ax, red);
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = sdx; part[2 * blockIdx.x + 1] = sx; }
    }
}

// ---------------------------------------------------------------------------
// Launchers: one instantiation per transform length (image sides 16 .. 8192).
#define PD_N_DISPATCH(n_, CALL)                                  \
    switch (n_) {                                                \
        case 16: { constexpr int NN = 16; CALL; } break;         \
        case 32: { constexpr int NN = 32; CALL; } break;         \
        case 64: { constexpr int NN = 64; CALL; } break;         \
        case 128: { constexpr int NN = 128; CALL; } break;       \
        case 256: { constexpr int NN = 256; CALL; } break;       \
        case 512: { constexpr int NN = 512; CALL; } break;       \
        case 1024: { constexpr int NN = 1024; CALL; } break;     \
        case 2048: { constexpr int NN = 2048; CALL; } break;     \
        case 4096: { constexpr int NN = 4096; CALL; } break;     \
        case 8192: { if constexpr (sizeof(R) == 4) { constexpr int NN = 8192; CALL; } \
                     else return cudaErrorInvalidValue; } break; \
        default: return cudaErrorInvalidValue;                   \
    }

// complex elements of one image's half-grid intermediates: t1 (ny rows) and F Z x (Ky rows)
static int64_t t1_elems(const pd_plan* p) { return (int64_t)(p->g.nx / 4 + 1) * 4 * p->g.ny; }
static int64_t gb_elems(const pd_plan* p) { return (int64_t)(p->g.nx / 4 + 1) * 4 * p->g.Ky; }

template <typename R, int N>
static cudaError_t launch_fwd_rows(const pd_plan* p, const R* x, cplx_t<R>* t1, int batch, cudaStream_t s) {
    using P = PassShape<R, N>;
    cudaError_t e;
    if ((e = ensure_smem(k_fwd_rows<R, N>, P::SMEM_ROWS))) return e;
    k_fwd_rows<R, N><<<dim3(p->g.ny / (2 * P::PAIRS), batch), P::NT_ROWS, P::SMEM_ROWS, s>>>(
        x, t1, (const R*)p->cx, (const R*)p->cy, (const cplx_t<R>*)p->twx, p->g.ny, t1_elems(p));
    return cudaGetLastError();
}
template <typename R, int N>
static cudaError_t launch_fwd_cols(const pd_plan* p, const cplx_t<R>* t1, cplx_t<R>* gb, int batch,
                                   cudaStream_t s) {
    using P = PassShape<R, N>;
    cudaError_t e;
    if ((e = ensure_smem(k_fwd_cols<R, N>, P::SMEM_COLS))) return e;
    k_fwd_cols<R, N><<<dim3((p->g.nx / 4 + 1) * (4 / P::CQ), batch), P::NT_COLS, P::SMEM_COLS, s>>>(
        t1, gb, (const cplx_t<R>*)p->twy, t1_elems(p), gb_elems(p));
    return cudaGetLastError();
}
template <typename R, int N>
static cudaError_t launch_inv_cols(const pd_plan* p, const cplx_t<R>* U, cplx_t<R>* t1, int batch,
                                   cudaStream_t s) {
    using P = PassShape<R, N>;
    cudaError_t e;
    if ((e = ensure_smem(k_inv_cols<R, N>, P::SMEM_COLS))) return e;
    k_inv_cols<R, N><<<dim3((p->g.nx / 4 + 1) * (4 / P::CQ), batch), P::NT_COLS, P::SMEM_COLS, s>>>(
        U, t1, (const cplx_t<R>*)p->twy, p->g.Kx, t1_elems(p));
    return cudaGetLastError();
}
template <typename R, int N>
static cudaError_t launch_inv_rows(const pd_plan* p, const cplx_t<R>* t1, R* out, const PrimalArgs* pa, int batch,
                                   cudaStream_t s) {
    using P = PassShape<R, N>;
    cudaError_t e;
    if ((e = ensure_smem(k_inv_rows<R, N>, P::SMEM_ROWS))) return e;
    const int ctas = p->g.ny / (2 * P::PAIRS);
    if (pa == nullptr)
        k_inv_rows<R, N><<<dim3(ctas, batch), P::NT_ROWS, P::SMEM_ROWS, s>>>(
            t1, out, (const R*)p->cx, (const R*)p->cy, (const cplx_t<R>*)p->twx, p->g.ny, 0, R(0), R(0), R(0),
            nullptr, nullptr, nullptr, nullptr, t1_elems(p));
    else
        k_inv_rows<R, N><<<ctas, P::NT_ROWS, P::SMEM_ROWS, s>>>(
            t1, nullptr, (const R*)p->cx, (const R*)p->cy, (const cplx_t<R>*)p->twx, p->g.ny, 1, (R)pa->tau,
            (R)pa->sigma, (R)pa->varsigma, (R*)pa->x, (R*)pa->xt, (const R*)pa->st, pa->part, t1_elems(p));
    return cudaGetLastError();
}

int inv_rows_ctas(const pd_plan* p) {
    int pairs = 1;
    auto get = [&](auto tag) {
        using R = decltype(tag);
        cudaError_t e = cudaSuccess;
        PD_N_DISPATCH(p->g.nx, (pairs = PassShape<R, NN>::PAIRS));
        return e;
    };
    if (p->prec == PD_F64) get(double{}); else get(float{});
    return p->g.ny / (2 * pairs);
}

template <typename R>
cudaError_t fwd_fft(const pd_plan* p, const R* x, cplx_t<R>* grid, cudaStream_t s, int batch, cplx_t<R>* t1) {
    cudaError_t e = cudaSuccess;
    if (!t1) t1 = (cplx_t<R>*)p->t1;
    prof_mark(PH_FWD_ROWS, 0, s);
    PD_N_DISPATCH(p->g.nx, (e = launch_fwd_rows<R, NN>(p, x, t1, batch, s)));
    prof_mark(PH_FWD_ROWS, 1, s);
    if (e) return e;
    prof_mark(PH_FWD_COLS, 0, s);
    PD_N_DISPATCH(p->g.ny, (e = launch_fwd_cols<R, NN>(p, t1, grid, batch, s)));
    prof_mark(PH_FWD_COLS, 1, s);
    return e;
}

template <typename R>
cudaError_t inv_fft(const pd_plan* p, const cplx_t<R>* grid, R* out, const PrimalArgs* pa, cudaStream_t s, int batch,
                    cplx_t<R>* t1) {
    cudaError_t e = cudaSuccess;
    if (!t1) t1 = (cplx_t<R>*)p->t1;
    prof_mark(PH_INV_COLS, 0, s);
    PD_N_DISPATCH(p->g.ny, (e = launch_inv_cols<R, NN>(p, grid, t1, batch, s)));
    prof_mark(PH_INV_COLS, 1, s);
    if (e) return e;
    prof_mark(PH_INV_ROWS, 0, s);
    PD_N_DISPATCH(p->g.nx, (e = launch_inv_rows<R, NN>(p, t1, out, pa, batch, s)));
    prof_mark(PH_INV_ROWS, 1, s);
    return e;
}

template cudaError_t fwd_fft<float>(const pd_plan*, const float*, float2*, cudaStream_t, int, float2*);
template cudaError_t fwd_fft<double>(const pd_plan*, const double*, double2*, cudaStream_t, int, double2*);
template cudaError_t inv_fft<float>(const pd_plan*, const float2*, float*, const PrimalArgs*, cudaStream_t, int,
                                    float2*);
template cudaError_t inv_fft<double>(const pd_plan*, const double2*, double*, const PrimalArgs*, cudaStream_t, int,
                                     double2*);

}  // namespace pdgb
