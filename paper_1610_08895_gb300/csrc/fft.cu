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

// One Stockham autosort stage of radix RAD over C = 2^logC interleaved sequences of
// length L held in shared memory s[l * C + c]. Each of the `nwork` worker threads owns
// E/RAD butterflies; values travel through registers, so the stage is in place. The
// first stage (Ns = 1, every twiddle 1) can take its inputs straight from global
// memory through ld(l, c) (GIN), and the last can hand its outputs to st(k, c, value,
// active) instead of shared memory (GOUT). st is called by every thread of the CTA, so
// it may exchange values between the lanes of a warp.
// threadIdx.x read through a volatile move, so the index arithmetic derived from it is
// redone per stage instead of being hoisted and held in registers across stages.
__device__ __forceinline__ int tid_here() {
    int t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
    return t;
}

template <typename R, int E, int RAD, int SIGN, bool GIN, bool GOUT, class Ld, class St>
__device__ __forceinline__ void stockham_stage(cplx_t<R>* s, int L, int logC, int Ns, const cplx_t<R>* tw2L,
                                               int nwork, const Ld& ld, const St& st) {
    using C2 = cplx_t<R>;
    constexpr int JOBS = E / RAD;
    const int tid = tid_here();
    const bool act = tid < nwork;
    const int LR = L / RAD;
    const int Cm = (1 << logC) - 1;
    const int twstep = (2 * L) / (Ns * RAD);
    C2 v[JOBS][RAD];
#pragma unroll
    for (int i = 0; i < JOBS; ++i) {
        const int q = tid + i * nwork;
        const int c = q & Cm, j = q >> logC;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            C2 a = mk<C2>(R(0), R(0));
            if (act) {
                if (GIN) {
                    a = ld(j + r * LR, c);
                } else {
                    a = s[((j + r * LR) << logC) + c];
                    if (r > 0 && Ns > 1) {
                        C2 w = tw2L[k * r * twstep];
                        if (SIGN > 0) w.y = -w.y;
                        a = cmul(a, w);
                    }
                }
            }
            v[i][r] = a;
        }
        dft_dif<RAD, SIGN>(v[i]);
    }
    if (!GIN && !GOUT) __syncthreads();
#pragma unroll
    for (int i = 0; i < JOBS; ++i) {
        const int q = tid + i * nwork;
        const int c = q & Cm, j = q >> logC;
        const int k = j & (Ns - 1);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            if (GOUT) st(base + r * Ns, c, v[i][bitrev<RAD>(r)], act);
            else if (act) s[((base + r * Ns) << logC) + c] = v[i][bitrev<RAD>(r)];
        }
    }
    if (!GOUT) __syncthreads();
}

template <typename R, int E, int RAD, int SIGN, bool GIN, bool GOUT, class Ld, class St>
__device__ __forceinline__ void first_stage(cplx_t<R>* s, int L, int logC, const cplx_t<R>* tw2L, int nwork,
                                            bool last, const Ld& ld, const St& st) {
    if (GOUT && last) stockham_stage<R, E, RAD, SIGN, GIN, GOUT>(s, L, logC, 1, tw2L, nwork, ld, st);
    else stockham_stage<R, E, RAD, SIGN, GIN, false>(s, L, logC, 1, tw2L, nwork, ld, st);
}

// C = 2^logC independent length-L DFTs (SIGN -1 forward, +1 inverse, unnormalised)
// with tw2L[k] = exp(-2 pi i k / (2L)). Inputs come from ld when GIN, else from s in
// natural order s[l * C + c]; outputs go to st when GOUT, else they are left in natural
// order in s. The odd-sized radix runs first, where all its twiddles are 1.
template <typename R, int E, int SIGN, bool GIN, bool GOUT, class Ld, class St>
__device__ void fft_io(cplx_t<R>* s, int L, int logC, const cplx_t<R>* tw2L, const Ld& ld, const St& st) {
    constexpr int LOGE = E >= 16 ? 4 : 3;
    constexpr int RB = 1 << LOGE;
    const int nwork = (L << logC) / E;
    const int bits = 31 - __clz(L);
    const int rem = bits % LOGE;
    const int nst = bits / LOGE + (rem ? 1 : 0);
    const bool last = nst == 1;
    if (rem == 3) first_stage<R, E, 8, SIGN, GIN, GOUT>(s, L, logC, tw2L, nwork, last, ld, st);
    else if (rem == 2) first_stage<R, E, 4, SIGN, GIN, GOUT>(s, L, logC, tw2L, nwork, last, ld, st);
    else if (rem == 1) first_stage<R, E, 2, SIGN, GIN, GOUT>(s, L, logC, tw2L, nwork, last, ld, st);
    else first_stage<R, E, RB, SIGN, GIN, GOUT>(s, L, logC, tw2L, nwork, last, ld, st);
    int Ns = rem ? 1 << rem : RB;
    for (int b = nst - 1; b > 0; --b) {
        if (GOUT && b == 1) stockham_stage<R, E, RB, SIGN, false, GOUT>(s, L, logC, Ns, tw2L, nwork, ld, st);
        else stockham_stage<R, E, RB, SIGN, false, false>(s, L, logC, Ns, tw2L, nwork, ld, st);
        Ns <<= LOGE;
    }
}

template <typename R> struct FftE;
template <> struct FftE<float> { static constexpr int value = 16; };
template <> struct FftE<double> { static constexpr int value = 8; };

template <typename C> __device__ __forceinline__ C shfl_xor(C v, int m) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
    return v;
}

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
    auto nl = [](int, int) { return mk<C2>(R(0), R(0)); };
    auto ns = [](int, int, C2, bool) {};
    fft_io<R, FftE<R>::value, -1, false, false>(s, nx, logC, twx, nl, ns);
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
    auto nl = [](int, int) { return mk<C2>(R(0), R(0)); };
    auto ns = [](int, int, C2, bool) {};
    fft_io<R, FftE<R>::value, -1, false, false>(s, ny, logC, twy, nl, ns);
    for (int e = threadIdx.x; e < Ky * CQ; e += blockDim.x) {
        const int ky = e / CQ, qq = e - ky * CQ;
        gb[((int64_t)p * Ky + ky) * 4 + q0 + qq] = s[(ky >> 1) * C + (ky & 1) * CQ + qq];
    }
}

// Inverse column pass (F^H along y, crop to ny rows). Sequence c = r CQ + qq holds the
// grid rows of parity r of column q0 + qq; the cropped row iy is
// E[m] + conj(W_2ny^lc) O[m] with lc = iy - ny/2, m = lc mod ny. DIRECT: the odd
// sequence's value comes from the lane CQ away and the row is stored from registers.
template <typename R, bool DIRECT>
__global__ void __launch_bounds__(1024) k_inv_cols(const cplx_t<R>* __restrict__ U, cplx_t<R>* __restrict__ t1,
                                                   const cplx_t<R>* __restrict__ twy, int ny, int CQ) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int C = 2 * CQ, logC = 31 - __clz(C), lq = logC - 1;
    const int Ky = 2 * ny, h = ny / 2;
    const int per = 4 / CQ;
    const int p = blockIdx.x / per, q0 = (blockIdx.x - p * per) * CQ;
    const C2* src = U + ((int64_t)p * Ky << 2) + q0;
    C2* dst = t1 + ((int64_t)p * ny << 2) + q0;
    auto ld = [&](int m, int c) { return src[((2 * m + (c >> lq)) << 2) + (c & (CQ - 1))]; };
    if (DIRECT) {
        auto st = [&](int k, int c, C2 v, bool act) {
            const C2 o = shfl_xor(v, CQ);
            if (act && !(c >> lq)) {
                const int lc = k < h ? k : k - ny;
                dst[((lc + h) << 2) + c] = cadd(v, cmul(cconj(twy[lc & (Ky - 1)]), o));
            }
        };
        fft_io<R, FftE<R>::value, +1, true, true>(s, ny, logC, twy, ld, st);
    } else {
        auto st = [](int, int, C2, bool) {};
        fft_io<R, FftE<R>::value, +1, true, false>(s, ny, logC, twy, ld, st);
        for (int e = threadIdx.x; e < ny * CQ; e += blockDim.x) {
            const int iy = e / CQ, qq = e - iy * CQ;
            const int lc = iy - h;
            const int m = lc & (ny - 1);
            const C2 w = cconj(twy[lc & (Ky - 1)]);
            dst[(iy << 2) + qq] = cadd(s[m * C + qq], cmul(w, s[m * C + CQ + qq]));
        }
    }
}

// Inverse row pass (F^H along x, crop, Re, deapodise), with either a plain store
// (mode 0) or the primal update of Alg. 1 steps 17-18 as epilogue (mode 1). Sequence
// c = 2 rho + r holds the grid columns of parity r of row iy0 + rho; DIRECT: the odd
// sequence's value comes from the neighbouring lane.
template <typename R, bool DIRECT>
__global__ void __launch_bounds__(1024) k_inv_rows(const cplx_t<R>* __restrict__ t1, R* __restrict__ out,
                                                   const R* __restrict__ cx, const R* __restrict__ cy,
                                                   const cplx_t<R>* __restrict__ twx, int nx, int ny, int RB,
                                                   int mode, R tau, R sigma, R varsigma, R* __restrict__ xs,
                                                   R* __restrict__ xt, const R* __restrict__ st_,
                                                   double* __restrict__ part) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    C2* s = reinterpret_cast<C2*>(smraw);
    const int C = 2 * RB, logC = 31 - __clz(C);
    const int Kx = 2 * nx, h = nx / 2;
    const int iy0 = blockIdx.x * RB;
    // per-thread partial sums of at most E terms in the working precision, then FP64
    R adx = R(0), ax = R(0);
    auto finish = [&](int iy, int ix, R g0) {
        const R g = g0 * cx[ix] * cy[iy];
        const int64_t idx = (int64_t)iy * nx + ix;
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
    };
    auto ld = [&](int m, int c) {
        const int kx = 2 * m + (c & 1);
        return t1[(((int64_t)(kx >> 2) * ny + iy0 + (c >> 1)) << 2) + (kx & 3)];
    };
    if (DIRECT) {
        auto st = [&](int k, int c, C2 v, bool act) {
            const C2 o = shfl_xor(v, 1);
            if (act && !(c & 1)) {
                const int lc = k < h ? k : k - nx;
                const C2 w = cconj(twx[lc & (Kx - 1)]);
                finish(iy0 + (c >> 1), lc + h, v.x + (w.x * o.x - w.y * o.y));
            }
        };
        fft_io<R, FftE<R>::value, +1, true, true>(s, nx, logC, twx, ld, st);
    } else {
        auto st = [](int, int, C2, bool) {};
        fft_io<R, FftE<R>::value, +1, true, false>(s, nx, logC, twx, ld, st);
        for (int e = threadIdx.x; e < RB * nx; e += blockDim.x) {
            const int rho = e / nx, ix = e - rho * nx;
            const int lc = ix - h;
            const int m = lc & (nx - 1);
            const C2 w = cconj(twx[lc & (Kx - 1)]);
            const C2 ev = s[m * C + 2 * rho], od = s[m * C + 2 * rho + 1];
            finish(iy0 + rho, ix, ev.x + (w.x * od.x - w.y * od.y));
        }
    }
    if (mode == 1) {
        const double sdx = block_sum((double)adx, red);
        const double sx = block_sum((double)ax, red);
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = sdx; part[2 * blockIdx.x + 1] = sx; }
    }
}

// ---------------------------------------------------------------------------
struct PassCfg {
    int rows_per_cta, cols_per_cta, threads_rows, threads_cols;
    size_t smem_rows, smem_cols;
    bool direct_rows, direct_cols;
};

template <typename R> static PassCfg pass_cfg(const pd_plan* p) {
    constexpr int E = FftE<R>::value;
    const int nx = p->g.nx, ny = p->g.ny;
    PassCfg c{};
    // at most 512 threads and 100 KB of shared memory per CTA, so two CTAs share an SM
    const int maxt = 512;
    const size_t maxs = 100 * 1024;
    int rb = 4;
    while (rb > 1 && (nx * 2 * rb / E > maxt || (size_t)nx * 2 * rb * sizeof(cplx_t<R>) > maxs)) rb >>= 1;
    int cq = 4;
    while (cq > 1 && (ny * 2 * cq / E > maxt || (size_t)ny * 2 * cq * sizeof(cplx_t<R>) > maxs)) cq >>= 1;
    if (rb > ny) rb = ny;
    c.rows_per_cta = rb;
    c.cols_per_cta = cq;
    auto thr = [](int work) { int t = ((work + 31) / 32) * 32; return t < 32 ? 32 : t; };
    c.threads_rows = thr(nx * 2 * rb / E);
    c.threads_cols = thr(ny * 2 * cq / E);
    c.smem_rows = (size_t)nx * 2 * rb * sizeof(cplx_t<R>);
    c.smem_cols = (size_t)ny * 2 * cq * sizeof(cplx_t<R>);
    // the register-level parity exchange of the inverse passes needs the partner
    // sequence in a fixed neighbouring lane for every butterfly job
    const int nw_rows = nx * 2 * rb / E, nw_cols = ny * 2 * cq / E;
    c.direct_rows = nx * 2 * rb >= E && nw_rows % 2 == 0;
    c.direct_cols = ny >= E && nw_cols % (2 * cq) == 0;
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

template <typename R, bool DR, bool DC>
static cudaError_t inv_fft_t(const pd_plan* p, const PassCfg& c, const cplx_t<R>* grid, R* out,
                             const PrimalArgs* pa, cudaStream_t s) {
    using C2 = cplx_t<R>;
    cudaError_t e;
    if ((e = ensure_smem(k_inv_cols<R, DC>, c.smem_cols))) return e;
    if ((e = ensure_smem(k_inv_rows<R, DR>, c.smem_rows))) return e;
    const int nx = p->g.nx, ny = p->g.ny;
    C2* t1 = (C2*)p->t1;
    prof_mark(PH_INV_COLS, 0, s);
    k_inv_cols<R, DC><<<(p->g.Kx / 4) * (4 / c.cols_per_cta), c.threads_cols, c.smem_cols, s>>>(
        grid, t1, (const C2*)p->twy, ny, c.cols_per_cta);
    prof_mark(PH_INV_COLS, 1, s);
    prof_mark(PH_INV_ROWS, 0, s);
    if (pa == nullptr) {
        k_inv_rows<R, DR><<<ny / c.rows_per_cta, c.threads_rows, c.smem_rows, s>>>(
            t1, out, (const R*)p->cx, (const R*)p->cy, (const C2*)p->twx, nx, ny, c.rows_per_cta, 0, R(0), R(0),
            R(0), nullptr, nullptr, nullptr, nullptr);
    } else {
        k_inv_rows<R, DR><<<ny / c.rows_per_cta, c.threads_rows, c.smem_rows, s>>>(
            t1, nullptr, (const R*)p->cx, (const R*)p->cy, (const C2*)p->twx, nx, ny, c.rows_per_cta, 1,
            (R)pa->tau, (R)pa->sigma, (R)pa->varsigma, (R*)pa->x, (R*)pa->xt, (const R*)pa->st, pa->part);
    }
    prof_mark(PH_INV_ROWS, 1, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t inv_fft(const pd_plan* p, const cplx_t<R>* grid, R* out, const PrimalArgs* pa, cudaStream_t s) {
    const PassCfg c = pass_cfg<R>(p);
    if (c.direct_rows && c.direct_cols) return inv_fft_t<R, true, true>(p, c, grid, out, pa, s);
    if (c.direct_rows) return inv_fft_t<R, true, false>(p, c, grid, out, pa, s);
    if (c.direct_cols) return inv_fft_t<R, false, true>(p, c, grid, out, pa, s);
    return inv_fft_t<R, false, false>(p, c, grid, out, pa, s);
}

template cudaError_t fwd_fft<float>(const pd_plan*, const float*, float2*, cudaStream_t);
template cudaError_t fwd_fft<double>(const pd_plan*, const double*, double2*, cudaStream_t);
template cudaError_t inv_fft<float>(const pd_plan*, const float2*, float*, const PrimalArgs*, cudaStream_t);
template cudaError_t inv_fft<double>(const pd_plan*, const double2*, double*, const PrimalArgs*, cudaStream_t);

}  // namespace pdgb
