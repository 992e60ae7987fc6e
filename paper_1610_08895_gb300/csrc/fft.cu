// Oversampled 2-D FFT passes of Phi = G F Z and of its adjoint (Sec. 2), as
// shared-memory Stockham transforms.
//
// The grid is (2 ny) x (2 nx) but only ny x nx of its input cells are non-zero
// (zero padding by Z), and the adjoint only needs ny x nx of its outputs (the
// crop of Z^T). Every pass therefore runs half-length transforms: with a length
// 2n transform split into even and odd outputs (forward) or inputs (inverse),
//   X[2j + r] = sum_l (x_l W_2n^{r l}) W_n^{j l},
//   x_l       = E_l + W_2n^{-l} O_l,  E/O = inverse length-n transforms of even/odd inputs,
// so each CTA transforms 2 x (columns it owns) sequences of length n in shared
// memory. Layouts: images are row-major [ny][nx]; the row-pass intermediate t1
// and the grids use column panels [K/4][rows][4] so that every column pass
// reads and writes contiguous slabs.
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

// One Stockham autosort stage of radix RAD over C interleaved sequences of length L
// held in shared memory s[l * C + c]. Each of the `nwork` worker threads owns E/RAD
// butterflies; values travel through registers, so the stage is in place.
template <typename R, int E, int RAD, int SIGN>
__device__ __forceinline__ void stockham_stage(cplx_t<R>* s, int L, int logC, int Ns, const cplx_t<R>* tw2L,
                                               int nwork) {
    using C2 = cplx_t<R>;
    constexpr int JOBS = E / RAD;
    const int tid = threadIdx.x;
    const int LR = L / RAD;
    const int Cm = (1 << logC) - 1;
    const int twstep = (2 * L) / (Ns * RAD);
    C2 v[JOBS][RAD];
    if (tid < nwork) {
#pragma unroll
        for (int i = 0; i < JOBS; ++i) {
            const int q = tid + i * nwork;
            const int c = q & Cm, j = q >> logC;
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                C2 a = s[((j + r * LR) << logC) + c];
                if (r > 0 && Ns > 1) {
                    C2 w = tw2L[k * r * twstep];
                    if (SIGN > 0) w.y = -w.y;
                    a = cmul(a, w);
                }
                v[i][r] = a;
            }
            dft_dif<RAD, SIGN>(v[i]);
        }
    }
    __syncthreads();
    if (tid < nwork) {
#pragma unroll
        for (int i = 0; i < JOBS; ++i) {
            const int q = tid + i * nwork;
            const int c = q & Cm, j = q >> logC;
            const int k = j & (Ns - 1);
            const int base = (j - k) * RAD + k;
#pragma unroll
            for (int r = 0; r < RAD; ++r) s[((base + r * Ns) << logC) + c] = v[i][bitrev<RAD>(r)];
        }
    }
    __syncthreads();
}

// C = 2^logC independent length-L DFTs (SIGN -1 forward, +1 inverse, unnormalised)
// on shared memory; tw2L[k] = exp(-2 pi i k / (2L)).
template <typename R, int E, int SIGN>
__device__ void fft_smem(cplx_t<R>* s, int L, int logC, const cplx_t<R>* tw2L) {
    const int nwork = (L << logC) / E;
    const int bits = 31 - __clz(L);
    constexpr int LOGE = E >= 16 ? 4 : 3;
    // the odd radix goes first, where every twiddle is 1 (Ns = 1)
    int rem = bits % LOGE;
    int Ns = 1;
    if (rem == 3) { stockham_stage<R, E, 8, SIGN>(s, L, logC, Ns, tw2L, nwork); Ns <<= 3; }
    else if (rem == 2) { stockham_stage<R, E, 4, SIGN>(s, L, logC, Ns, tw2L, nwork); Ns <<= 2; }
    else if (rem == 1) { stockham_stage<R, E, 2, SIGN>(s, L, logC, Ns, tw2L, nwork); Ns <<= 1; }
    for (int b = bits - rem; b > 0; b -= LOGE) {
        stockham_stage<R, E, (E >= 16 ? 16 : 8), SIGN>(s, L, logC, Ns, tw2L, nwork);
        Ns <<= LOGE;
    }
}

template <typename R> struct FftE;
template <> struct FftE<float> { static constexpr int value = 16; };
template <> struct FftE<double> { static constexpr int value = 8; };

// ---------------------------------------------------------------------------
// Forward row pass (Z then F along x): RB image rows per CTA; smem column 2*rho + r
// holds row rho pre-twiddled for the even (r = 0) or odd (r = 1) outputs.
template <typename R>
__global__ void __launch_bounds__(1024) k_fwd_rows(const R* __restrict__ x, cplx_t<R>* __restrict__ t1,
                                                   const R* __restrict__ cx, const R* __restrict__ cy,
                                                   const cplx_t<R>* __restrict__ twx, int nx, int ny, int RB) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int logC = 31 - __clz(2 * RB), C = 2 * RB;
    const int Kx = 2 * nx;
    const int iy0 = blockIdx.x * RB;
    for (int e = threadIdx.x; e < RB * nx; e += blockDim.x) {
        const int rho = e / nx, ix = e - rho * nx;
        const int iy = iy0 + rho;
        const R val = x[(int64_t)iy * nx + ix] * cx[ix] * cy[iy];
        const int lc = ix - nx / 2;
        const int m = lc & (nx - 1);
        const C2 w = twx[lc & (Kx - 1)];
        s[m * C + 2 * rho] = mk<C2>(val, R(0));
        s[m * C + 2 * rho + 1] = mk<C2>(val * w.x, val * w.y);
    }
    __syncthreads();
    fft_smem<R, FftE<R>::value, -1>(s, nx, logC, twx);
    for (int e = threadIdx.x; e < RB * Kx; e += blockDim.x) {
        const int p = e / (4 * RB), rem = e - p * 4 * RB;
        const int rho = rem >> 2, q = rem & 3;
        const int kx = 4 * p + q;
        t1[((int64_t)p * ny + iy0 + rho) * 4 + q] = s[(kx >> 1) * C + 2 * rho + (kx & 1)];
    }
}

// Forward column pass (F along y): CQ columns of one panel per CTA; smem column
// r * CQ + qq holds column qq pre-twiddled for output parity r.
template <typename R>
__global__ void __launch_bounds__(1024) k_fwd_cols(const cplx_t<R>* __restrict__ t1, cplx_t<R>* __restrict__ gb,
                                                   const cplx_t<R>* __restrict__ twy, int ny, int CQ) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int C = 2 * CQ, logC = 31 - __clz(C);
    const int Ky = 2 * ny;
    const int per = 4 / CQ;
    const int p = blockIdx.x / per, q0 = (blockIdx.x - p * per) * CQ;
    for (int e = threadIdx.x; e < ny * CQ; e += blockDim.x) {
        const int iy = e / CQ, qq = e - iy * CQ;
        const C2 val = t1[((int64_t)p * ny + iy) * 4 + q0 + qq];
        const int lc = iy - ny / 2;
        const int m = lc & (ny - 1);
        s[m * C + qq] = val;
        s[m * C + CQ + qq] = cmul(val, twy[lc & (Ky - 1)]);
    }
    __syncthreads();
    fft_smem<R, FftE<R>::value, -1>(s, ny, logC, twy);
    for (int e = threadIdx.x; e < Ky * CQ; e += blockDim.x) {
        const int ky = e / CQ, qq = e - ky * CQ;
        gb[((int64_t)p * Ky + ky) * 4 + q0 + qq] = s[(ky >> 1) * C + (ky & 1) * CQ + qq];
    }
}

// Inverse column pass (F^H along y, crop to ny rows).
template <typename R>
__global__ void __launch_bounds__(1024) k_inv_cols(const cplx_t<R>* __restrict__ U, cplx_t<R>* __restrict__ t1,
                                                   const cplx_t<R>* __restrict__ twy, int ny, int CQ) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int C = 2 * CQ, logC = 31 - __clz(C);
    const int Ky = 2 * ny;
    const int per = 4 / CQ;
    const int p = blockIdx.x / per, q0 = (blockIdx.x - p * per) * CQ;
    for (int e = threadIdx.x; e < Ky * CQ; e += blockDim.x) {
        const int ky = e / CQ, qq = e - ky * CQ;
        s[(ky >> 1) * C + (ky & 1) * CQ + qq] = U[((int64_t)p * Ky + ky) * 4 + q0 + qq];
    }
    __syncthreads();
    fft_smem<R, FftE<R>::value, +1>(s, ny, logC, twy);
    for (int e = threadIdx.x; e < ny * CQ; e += blockDim.x) {
        const int iy = e / CQ, qq = e - iy * CQ;
        const int lc = iy - ny / 2;
        const int m = lc & (ny - 1);
        const C2 w = cconj(twy[lc & (Ky - 1)]);
        t1[((int64_t)p * ny + iy) * 4 + q0 + qq] = cadd(s[m * C + qq], cmul(w, s[m * C + CQ + qq]));
    }
}

// Inverse row pass (F^H along x, crop, Re, deapodise), with either a plain store
// (mode 0) or the primal update of Alg. 1 steps 17-18 as epilogue (mode 1).
template <typename R>
__global__ void __launch_bounds__(1024) k_inv_rows(const cplx_t<R>* __restrict__ t1, R* __restrict__ out,
                                                   const R* __restrict__ cx, const R* __restrict__ cy,
                                                   const cplx_t<R>* __restrict__ twx, int nx, int ny, int RB,
                                                   int mode, R tau, R sigma, R varsigma, R* __restrict__ xs,
                                                   R* __restrict__ xt, const R* __restrict__ st,
                                                   double* __restrict__ part) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int C = 2 * RB, logC = 31 - __clz(C);
    const int Kx = 2 * nx;
    const int iy0 = blockIdx.x * RB;
    for (int e = threadIdx.x; e < RB * Kx; e += blockDim.x) {
        const int p = e / (4 * RB), rem = e - p * 4 * RB;
        const int rho = rem >> 2, q = rem & 3;
        const int kx = 4 * p + q;
        s[(kx >> 1) * C + 2 * rho + (kx & 1)] = t1[((int64_t)p * ny + iy0 + rho) * 4 + q];
    }
    __syncthreads();
    fft_smem<R, FftE<R>::value, +1>(s, nx, logC, twx);
    double adx = 0.0, ax = 0.0;
    for (int e = threadIdx.x; e < RB * nx; e += blockDim.x) {
        const int rho = e / nx, ix = e - rho * nx;
        const int iy = iy0 + rho;
        const int lc = ix - nx / 2;
        const int m = lc & (nx - 1);
        const C2 w = cconj(twx[lc & (Kx - 1)]);
        const C2 ev = s[m * C + 2 * rho], od = s[m * C + 2 * rho + 1];
        const R g = (ev.x + (w.x * od.x - w.y * od.y)) * cx[ix] * cy[iy];
        const int64_t idx = (int64_t)iy * nx + ix;
        if (mode == 0) {
            out[idx] = g;
        } else {
            const R xo = xs[idx];
            R xn = xo - tau * (sigma * st[idx] + varsigma * g);
            xn = xn > R(0) ? xn : R(0);
            xt[idx] = R(2) * xn - xo;
            xs[idx] = xn;
            const double dd = (double)xn - (double)xo;
            adx += dd * dd;
            ax += (double)xn * (double)xn;
        }
    }
    if (mode == 1) {
        const double sdx = block_sum(adx, red);
        const double sx = block_sum(ax, red);
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = sdx; part[2 * blockIdx.x + 1] = sx; }
    }
}

// ---------------------------------------------------------------------------
struct PassCfg { int rows_per_cta, cols_per_cta, threads_rows, threads_cols; size_t smem_rows, smem_cols; };

template <typename R> static PassCfg pass_cfg(const pd_plan* p) {
    constexpr int E = FftE<R>::value;
    const int nx = p->g.nx, ny = p->g.ny;
    PassCfg c{};
    // at most 100 KB of shared memory and 512 threads per CTA, so two CTAs share an SM
    // and one CTA's loads overlap the other's butterflies
    int rb = 4;
    while (rb > 1 && (nx * 2 * rb / E > 512 || (size_t)nx * 2 * rb * sizeof(cplx_t<R>) > 100 * 1024)) rb >>= 1;
    int cq = 4;
    while (cq > 1 && (ny * 2 * cq / E > 512 || (size_t)ny * 2 * cq * sizeof(cplx_t<R>) > 100 * 1024)) cq >>= 1;
    if (rb > ny) rb = ny;
    c.rows_per_cta = rb;
    c.cols_per_cta = cq;
    auto thr = [](int work) { int t = ((work + 31) / 32) * 32; return t < 32 ? 32 : t; };
    c.threads_rows = thr(nx * 2 * rb / E);
    c.threads_cols = thr(ny * 2 * cq / E);
    c.smem_rows = (size_t)nx * 2 * rb * sizeof(cplx_t<R>);
    c.smem_cols = (size_t)ny * 2 * cq * sizeof(cplx_t<R>);
    return c;
}

int inv_rows_ctas(const pd_plan* p) {
    PassCfg c = p->prec == PD_F64 ? pass_cfg<double>(p) : pass_cfg<float>(p);
    return p->g.ny / c.rows_per_cta;
}

template <typename R>
cudaError_t fwd_fft(const pd_plan* p, const R* x, cplx_t<R>* grid, cudaStream_t s) {
    using C2 = cplx_t<R>;
    const PassCfg c = pass_cfg<R>(p);
    cudaError_t e;
    if ((e = ensure_smem(k_fwd_rows<R>, c.smem_rows))) return e;
    if ((e = ensure_smem(k_fwd_cols<R>, c.smem_cols))) return e;
    const int nx = p->g.nx, ny = p->g.ny;
    C2* t1 = (C2*)p->t1;
    prof_mark(PH_FWD_ROWS, 0, s);
    k_fwd_rows<R><<<ny / c.rows_per_cta, c.threads_rows, c.smem_rows, s>>>(
        x, t1, (const R*)p->cx, (const R*)p->cy, (const C2*)p->twx, nx, ny, c.rows_per_cta);
    prof_mark(PH_FWD_ROWS, 1, s);
    prof_mark(PH_FWD_COLS, 0, s);
    k_fwd_cols<R><<<(p->g.Kx / 4) * (4 / c.cols_per_cta), c.threads_cols, c.smem_cols, s>>>(
        t1, grid, (const C2*)p->twy, ny, c.cols_per_cta);
    prof_mark(PH_FWD_COLS, 1, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t inv_fft(const pd_plan* p, const cplx_t<R>* grid, R* out, const PrimalArgs* pa, cudaStream_t s) {
    using C2 = cplx_t<R>;
    const PassCfg c = pass_cfg<R>(p);
    cudaError_t e;
    if ((e = ensure_smem(k_inv_cols<R>, c.smem_cols))) return e;
    if ((e = ensure_smem(k_inv_rows<R>, c.smem_rows))) return e;
    const int nx = p->g.nx, ny = p->g.ny;
    C2* t1 = (C2*)p->t1;
    prof_mark(PH_INV_COLS, 0, s);
    k_inv_cols<R><<<(p->g.Kx / 4) * (4 / c.cols_per_cta), c.threads_cols, c.smem_cols, s>>>(
        grid, t1, (const C2*)p->twy, ny, c.cols_per_cta);
    prof_mark(PH_INV_COLS, 1, s);
    prof_mark(PH_INV_ROWS, 0, s);
    if (pa == nullptr) {
        k_inv_rows<R><<<ny / c.rows_per_cta, c.threads_rows, c.smem_rows, s>>>(
            t1, out, (const R*)p->cx, (const R*)p->cy, (const C2*)p->twx, nx, ny, c.rows_per_cta, 0, R(0), R(0),
            R(0), nullptr, nullptr, nullptr, nullptr);
    } else {
        k_inv_rows<R><<<ny / c.rows_per_cta, c.threads_rows, c.smem_rows, s>>>(
            t1, nullptr, (const R*)p->cx, (const R*)p->cy, (const C2*)p->twx, nx, ny, c.rows_per_cta, 1,
            (R)pa->tau, (R)pa->sigma, (R)pa->varsigma, (R*)pa->x, (R*)pa->xt, (const R*)pa->st, pa->part);
    }
    prof_mark(PH_INV_ROWS, 1, s);
    return cudaGetLastError();
}

template cudaError_t fwd_fft<float>(const pd_plan*, const float*, float2*, cudaStream_t);
template cudaError_t fwd_fft<double>(const pd_plan*, const double*, double2*, cudaStream_t);
template cudaError_t inv_fft<float>(const pd_plan*, const float2*, float*, const PrimalArgs*, cudaStream_t);
template cudaError_t inv_fft<double>(const pd_plan*, const double2*, double*, const PrimalArgs*, cudaStream_t);

}  // namespace pdgb
