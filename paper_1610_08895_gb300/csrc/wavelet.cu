// Sparsity dictionary Psi = b^{-1/2} [Psi_1 ... Psi_b] (Sec. 3: a collection of b
// bases, the Dirac basis and Daubechies wavelets db1..db8), and the sparsity dual
// update of Algorithm 1 steps 13-14.
//
// Periodic separable filter banks: analysis a_k = sum_j h_j x_{(2k+j) mod m},
// d_k = sum_j g_j x_{(2k+j) mod m}, g_j = (-1)^j h_{L-1-j}; rows then columns;
// L levels in the packed layout (coarsest approximation top-left). Synthesis is
// the transpose. Each CTA stages one input tile plus its filter halo in shared
// memory, filters rows then columns there, and writes the four sub-bands.
//
// Step 13 is s <- s + w - S_alpha(s + w) = clip(s + w, -alpha, alpha) (Moreau,
// eq. prox-L1), fused into the analysis epilogue; the change ds = s_new - s_old
// is synthesised and added to s~ (step 14) so that inactive bases cost nothing.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"
#include "host_math.hpp"
#include "plan.hpp"

namespace pdgb {

constexpr int AT = 32;   // analysis output tile edge (per sub-band)
constexpr int ST = 64;   // synthesis output tile edge
constexpr int NT_W = 256;

template <typename R> __device__ __forceinline__ R clip(R v, R a) { return v > a ? a : (v < -a ? -a : v); }

// -------------------------------------------------------------------- analysis
// The filter pair of one basis in registers: h (low-pass) and g_j = (-1)^j h_{LF-1-j}.
template <typename R, int LF>
__device__ __forceinline__ void load_filters(const R* __restrict__ filt, int k, R* h, R* g) {
#pragma unroll
    for (int j = 0; j < LF; ++j) {
        h[j] = filt[k * MAX_FILTER + j];
        g[j] = ((j & 1) ? R(-1) : R(1)) * filt[k * MAX_FILTER + LF - 1 - j];
    }
}

// Dispatch on the filter length of basis k (2, 4, ..., 16: db1 .. db8) to a body with the
// length as a compile-time constant (fully unrolled taps, filters in registers).
#define PD_LF_DISPATCH(lf_, CALL)                           \
    switch (lf_) {                                          \
        case 2: { constexpr int LF = 2; CALL; } break;      \
        case 4: { constexpr int LF = 4; CALL; } break;      \
        case 6: { constexpr int LF = 6; CALL; } break;      \
        case 8: { constexpr int LF = 8; CALL; } break;      \
        case 10: { constexpr int LF = 10; CALL; } break;    \
        case 12: { constexpr int LF = 12; CALL; } break;    \
        case 14: { constexpr int LF = 14; CALL; } break;    \
        default: { constexpr int LF = 16; CALL; } break;    \
    }

constexpr int ARB = 4;   // analysis outputs per thread along a row (row pass) or column (column pass)

// One analysis level of basis k on an output tile of ty x tx per sub-band at (oy0, ox0)
// of the (my x mx) region. Staged input rows have an odd pitch IWP and the row-pass
// results a pitch tx + 1, so that threads walking down a column hit distinct banks.
// Row pass: a thread computes ARB consecutive outputs of one input row from
// LF + 2 ARB - 2 staged values (consecutive threads take consecutive rows); column
// pass: ARB consecutive output rows of one column, the low-pass half (LL, LH) and then
// the high-pass half (HL, HH). MODE 0 writes the scaled coefficients, MODE 1 the
// step-13 update of s and its change ds.
template <typename R, int MODE, int LF>
__device__ __forceinline__ void dwt_body(const R* __restrict__ src, R* __restrict__ ll_out, R* __restrict__ out,
                                         R* __restrict__ ds, const R* __restrict__ wt, const R* __restrict__ filt,
                                         int k, int my, int mx,
                                         int oy0, int ox0, int ty, int tx, bool last, int64_t boff, int nx,
                                         int64_t ll_off, R scale, R alpha, R* sm) {
    constexpr int NX = LF + 2 * ARB - 2;               // staged values per ARB outputs
    const int hy = my >> 1, hx = mx >> 1;
    const int IH = 2 * ty + LF - 2, IW = 2 * tx + LF - 2, IWP = IW | 1, TP = tx + 1;
    R* in = sm;                                        // [IH][IWP]
    R* ra = in + IH * IWP;                             // [IH][TP]
    R* rd = ra + IH * TP;                              // [IH][TP]
    R h[LF], g[LF];
    load_filters<R, LF>(filt, k, h, g);
    stage_batched<8>(in, IH * IWP, [&](int i) {
        const int r = i / IWP, cc = i - r * IWP;
        const int gy = (2 * oy0 + r) & (my - 1), gx = (2 * ox0 + cc) & (mx - 1);
        return src[(int64_t)gy * mx + gx];
    });
    __syncthreads();
    // row pass
    const int nrg = (tx + ARB - 1) / ARB;
    for (int it = threadIdx.x; it < IH * nrg; it += blockDim.x) {
        const int r = it % IH, c0 = (it / IH) * ARB;
        const R* row = in + r * IWP + 2 * c0;
        R x[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = (2 * c0 + i < IWP) ? row[i] : R(0);
#pragma unroll
        for (int o = 0; o < ARB; ++o) {
            R a = 0, d = 0;
#pragma unroll
            for (int j = 0; j < LF; ++j) { a += h[j] * x[2 * o + j]; d += g[j] * x[2 * o + j]; }
            if (c0 + o < tx) { ra[r * TP + c0 + o] = a; rd[r * TP + c0 + o] = d; }
        }
    }
    __syncthreads();
    // column pass: rows r0 .. r0 + ARB - 1 of column c
    const int ncg = (ty + ARB - 1) / ARB;
    for (int item = threadIdx.x; item < ncg * tx; item += blockDim.x) {
        const int c = item % tx, r0 = (item / tx) * ARB;
        const int ox = ox0 + c;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            // half 0: the low-pass rows (LL, LH); half 1: the high-pass rows (HL, HH)
            const R* rr = half ? rd : ra;
            R sold[ARB][2];
            if (MODE == 1) {
#pragma unroll
                for (int o = 0; o < ARB; ++o) {
                    const int oy = oy0 + r0 + o;
                    if (r0 + o < ty) {
                        sold[o][0] = half ? out[boff + (int64_t)oy * nx + hx + ox]
                                          : (last ? out[boff + (int64_t)oy * nx + ox] : R(0));
                        sold[o][1] = out[boff + (int64_t)(hy + oy) * nx + (half ? hx : 0) + ox];
                    }
                }
            }
            R v[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) v[i] = 2 * r0 + i < IH ? rr[(2 * r0 + i) * TP + c] : R(0);
#pragma unroll
            for (int o = 0; o < ARB; ++o) {
                if (r0 + o >= ty) break;
                R lo = 0, hi = 0;
#pragma unroll
                for (int j = 0; j < LF; ++j) { lo += h[j] * v[2 * o + j]; hi += g[j] * v[2 * o + j]; }
                const int oy = oy0 + r0 + o;
                // low-pass along y: LL (half 0) or HL (half 1); high-pass along y: LH or HH
                const int64_t p_lo = boff + (int64_t)oy * nx + (half ? hx : 0) + ox;
                const int64_t p_hi = boff + (int64_t)(hy + oy) * nx + (half ? hx : 0) + ox;
                const bool store_lo = half || last;
                if (MODE == 0) {
                    if (store_lo) out[p_lo] = lo * scale;
                    out[p_hi] = hi * scale;
                } else {
                    // weighted prior: the threshold of each coefficient is alpha times its weight
                    if (store_lo) {
                        const R so = sold[o][0], sn = clip(so + lo * scale, wt ? alpha * wt[p_lo] : alpha);
                        out[p_lo] = sn; ds[p_lo] = sn - so;
                    }
                    const R so = sold[o][1], sn = clip(so + hi * scale, wt ? alpha * wt[p_hi] : alpha);
                    out[p_hi] = sn; ds[p_hi] = sn - so;
                }
                if (!half && !last) ll_out[ll_off + (int64_t)oy * hx + ox] = lo;
            }
        }
    }
}

// One level for every basis in blockIdx.z. MODE 0: out = coefficient * scale.
// MODE 1: s/ds update of step 13 (wt: per-coefficient weights of the reweighted prior,
// same layout as s, or null). The last level also treats the approximation band.
template <typename R, int MODE>
__global__ void __launch_bounds__(NT_W, 3) k_dwt_level(const R* __restrict__ x0, const R* __restrict__ ll_in,
                                                    R* __restrict__ ll_out, R* __restrict__ out, R* __restrict__ ds,
                                                    const R* __restrict__ wt,
                                                    const R* __restrict__ filt, const int32_t* __restrict__ flen,
                                                    const int32_t* __restrict__ active, int level, int L, int ny,
                                                    int nx, R scale, R alpha) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = blockIdx.z;
    const int lf = flen[k];
    if (lf == 0) return;                               // Dirac basis: separate kernel
    if (MODE == 1 && !active[k]) return;
    const int my = ny >> level, mx = nx >> level;
    const int hy = my >> 1, hx = mx >> 1;
    const int ty = min(AT, hy), tx = min(AT, hx);
    const int oy0 = blockIdx.y * ty, ox0 = blockIdx.x * tx;
    if (oy0 >= hy || ox0 >= hx) return;
    const R* src = level == 0 ? x0 : ll_in + (int64_t)k * (ny / 2) * (nx / 2);
    const int64_t boff = (int64_t)k * ny * nx, ll_off = (int64_t)k * (ny / 2) * (nx / 2);
    const bool last = level == L - 1;
    R* sm = reinterpret_cast<R*>(smraw);
    PD_LF_DISPATCH(lf, (dwt_body<R, MODE, LF>(src, ll_out, out, ds, wt, filt, k, my, mx, oy0, ox0, ty, tx, last, boff,
                                              nx, ll_off, scale, alpha, sm)));
}

// Dirac basis (identity): MODE 0 copies x * scale, MODE 1 applies step 13 elementwise.
template <typename R, int MODE>
__global__ void k_dirac(const R* __restrict__ x, R* __restrict__ out, R* __restrict__ ds,
                        const R* __restrict__ wt, const int32_t* __restrict__ flen,
                        const int32_t* __restrict__ active, int b, int64_t n, R scale, R alpha) {
    for (int k = 0; k < b; ++k) {
        if (flen[k] != 0 || (MODE == 1 && !active[k])) continue;
        R* o = out + (int64_t)k * n;
        R* d = ds + (int64_t)k * n;
        const R* wk = wt ? wt + (int64_t)k * n : nullptr;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            if (MODE == 0) {
                o[i] = x[i] * scale;
            } else {
                const R so = o[i], sn = clip(so + x[i] * scale, wk ? alpha * wk[i] : alpha);
                o[i] = sn;
                d[i] = sn - so;
            }
        }
    }
}

// -------------------------------------------------------------------- synthesis
constexpr int SRP = 2;   // synthesis: output row pairs per thread (column pass), column pairs (row pass)

// Reconstruct a (ty x tx) tile of the level-`level` region (size my x mx) of basis k from
// its four sub-bands; the approximation band comes from ll_in (or from the packed
// coefficients at the coarsest level). Result left in `res` (shared, [ty][tx + 1]).
// Output rows 2m and 2m + 1 both read the sub-band rows m + off - i, i < LF/2 (even and
// odd taps): a thread computes SRP row pairs of one column from LF/2 + SRP - 1 staged
// values per band; the row pass likewise along the rows.
template <typename R, int LF>
__device__ __forceinline__ void synth_tile(const R* __restrict__ coef, const R* __restrict__ ll_in,
                                           const R* __restrict__ filt, int k, int level, int L, int ny, int nx,
                                           int oy0, int ox0, int ty, int tx, R* sm, R* res) {
    constexpr int NV = LF / 2 + SRP - 1, OFF = LF / 2 - 1;
    const int my = ny >> level, mx = nx >> level;
    const int hy = my >> 1, hx = mx >> 1;
    const int NKy = ty / 2 + LF / 2 - 1, NKx = tx / 2 + LF / 2 - 1;
    const int kby = oy0 / 2 - LF / 2 + 1, kbx = ox0 / 2 - LF / 2 + 1;
    R* LLs = sm;                      // [NKy][NKx] x4 sub-bands
    R* HLs = LLs + NKy * NKx;
    R* LHs = HLs + NKy * NKx;
    R* HHs = LHs + NKy * NKx;
    const int NKP = NKx | 1;          // odd pitch: threads walking down a column hit distinct banks
    R* lo = HHs + NKy * NKx;          // [ty][NKP] columns synthesised, low-x half
    R* hi = lo + ty * NKP;
    R h[LF], g[LF];
    load_filters<R, LF>(filt, k, h, g);
    const int64_t boff = (int64_t)k * ny * nx;
    const bool coarsest = level == L - 1;
    const R* llsrc = ll_in + (int64_t)k * (ny / 2) * (nx / 2);
    constexpr int UB = 2;                 // rows of the strided loop whose loads go out together
    for (int base = threadIdx.x; base < NKy * NKx; base += UB * (int)blockDim.x) {
        R v[UB][4];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = base + u * (int)blockDim.x;
            if (i < NKy * NKx) {
                const int r = i / NKx, c = i - r * NKx;
                const int gy = (kby + r) & (hy - 1), gx = (kbx + c) & (hx - 1);
                v[u][0] = coarsest ? coef[boff + (int64_t)gy * nx + gx] : llsrc[(int64_t)gy * hx + gx];
                v[u][1] = coef[boff + (int64_t)gy * nx + hx + gx];
                v[u][2] = coef[boff + (int64_t)(hy + gy) * nx + gx];
                v[u][3] = coef[boff + (int64_t)(hy + gy) * nx + hx + gx];
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = base + u * (int)blockDim.x;
            if (i < NKy * NKx) { LLs[i] = v[u][0]; HLs[i] = v[u][1]; LHs[i] = v[u][2]; HHs[i] = v[u][3]; }
        }
    }
    __syncthreads();
    // column pass: rows 2m .. 2m + 2 SRP - 1 of column c of lo and hi
    const int npr = (ty / 2 + SRP - 1) / SRP;
    for (int it = threadIdx.x; it < npr * NKx; it += blockDim.x) {
        const int c = it % NKx, m0 = (it / NKx) * SRP;
        R a[4][NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int kk = m0 + OFF - (LF / 2 - 1) + i;      // sub-band rows m0 + OFF - (LF/2 - 1) ...
            const bool ok = kk < NKy;
            a[0][i] = ok ? LLs[kk * NKx + c] : R(0);
            a[1][i] = ok ? LHs[kk * NKx + c] : R(0);
            a[2][i] = ok ? HLs[kk * NKx + c] : R(0);
            a[3][i] = ok ? HHs[kk * NKx + c] : R(0);
        }
#pragma unroll
        for (int pq = 0; pq < SRP; ++pq) {
            const int m = m0 + pq;
            if (2 * m >= ty) break;
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                R l = 0, hh = 0;
#pragma unroll
                for (int i = 0; i < LF / 2; ++i) {
                    // tap j = 2 i + par reads sub-band row m + OFF - i = a[.][pq + LF/2 - 1 - i]
                    const int j = 2 * i + par, q = pq + LF / 2 - 1 - i;
                    l += h[j] * a[0][q] + g[j] * a[1][q];
                    hh += h[j] * a[2][q] + g[j] * a[3][q];
                }
                lo[(2 * m + par) * NKP + c] = l;
                hi[(2 * m + par) * NKP + c] = hh;
            }
        }
    }
    __syncthreads();
    // row pass: columns 2m .. 2m + 2 SRP - 1 of row r (consecutive threads take consecutive rows)
    const int npc = (tx / 2 + SRP - 1) / SRP;
    for (int it = threadIdx.x; it < ty * npc; it += blockDim.x) {
        const int r = it % ty, m0 = (it / ty) * SRP;
        R bl[NV], bh[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int kk = m0 + i;
            bl[i] = kk < NKx ? lo[r * NKP + kk] : R(0);
            bh[i] = kk < NKx ? hi[r * NKP + kk] : R(0);
        }
#pragma unroll
        for (int pq = 0; pq < SRP; ++pq) {
            const int m = m0 + pq;
            if (2 * m >= tx) break;
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                R v = 0;
#pragma unroll
                for (int i = 0; i < LF / 2; ++i) {
                    const int j = 2 * i + par, q = pq + LF / 2 - 1 - i;
                    v += h[j] * bl[q] + g[j] * bh[q];
                }
                res[r * (tx + 1) + 2 * m + par] = v;
            }
        }
    }
    __syncthreads();
}

// One level of one basis per blockIdx.z: reconstruct the (ny>>level) x (nx>>level)
// approximation of the next finer level into ll_out + basis * out_stride (at level 0:
// the basis's full-size synthesis).
template <typename R>
__global__ void __launch_bounds__(NT_W) k_idwt_level(const R* __restrict__ coef, const R* __restrict__ ll_in,
                                                     R* __restrict__ ll_out, const R* __restrict__ filt,
                                                     const int32_t* __restrict__ flen,
                                                     const int32_t* __restrict__ active, int level, int L, int ny,
                                                     int nx, int64_t out_stride) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = blockIdx.z;
    const int lf = flen[k];
    if (lf == 0) return;
    if (active && !active[k]) return;
    const int my = ny >> level, mx = nx >> level;
    const int ty = min(ST, my), tx = min(ST, mx);
    const int oy0 = blockIdx.y * ty, ox0 = blockIdx.x * tx;
    if (oy0 >= my || ox0 >= mx) return;
    R* sm = reinterpret_cast<R*>(smraw);
    R* res = sm + 4 * (ty / 2 + MAX_FILTER / 2) * (tx / 2 + MAX_FILTER / 2) + 2 * ty * ((tx / 2 + MAX_FILTER / 2) | 1);
    PD_LF_DISPATCH(lf, (synth_tile<R, LF>(coef, ll_in, filt, k, level, L, ny, nx, oy0, ox0, ty, tx, sm, res)));
    R* dst = ll_out + (int64_t)k * out_stride;
    for (int i = threadIdx.x; i < ty * tx; i += blockDim.x) {
        const int r = i / tx, c = i - r * tx;
        dst[(int64_t)(oy0 + r) * mx + ox0 + c] = res[r * (tx + 1) + c];
    }
}

// Sum of the bases' level-0 syntheses (the Dirac basis is its coefficients) over the
// active bases in basis order: MODE 0: out = acc * scale, MODE 1: out += acc * scale
// (the s~ update of step 14). Four consecutive pixels per thread.
template <typename R> struct Quad { R a, b, c, d; };
template <typename R> __device__ __forceinline__ Quad<R> ldq(const R* p) {
    if constexpr (sizeof(R) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        return {q.x, q.y, q.z, q.w};
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
        return {q0.x, q0.y, q1.x, q1.y};
    }
}
template <typename R> __device__ __forceinline__ void stq(R* p, const Quad<R>& v) {
    if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v.a, v.b, v.c, v.d);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(v.a, v.b);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v.c, v.d);
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_syn_sum(const R* __restrict__ coef, const R* __restrict__ part,
                                                 const int32_t* __restrict__ flen, const int32_t* __restrict__ active,
                                                 int b, int64_t n, R* __restrict__ out, R scale) {
    for (int64_t i4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 4 * i4 < n; i4 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = 4 * i4;
        Quad<R> acc{R(0), R(0), R(0), R(0)};
        for (int k = 0; k < b; ++k) {
            if (MODE == 1 && !active[k]) continue;
            const Quad<R> v = ldq((flen[k] == 0 ? coef : part) + (int64_t)k * n + i);
            acc.a += v.a; acc.b += v.b; acc.c += v.c; acc.d += v.d;
        }
        Quad<R> o{acc.a * scale, acc.b * scale, acc.c * scale, acc.d * scale};
        if (MODE == 1) {
            const Quad<R> prev = ldq(out + i);
            o.a += prev.a; o.b += prev.b; o.c += prev.c; o.d += prev.d;
        }
        stq(out + i, o);
    }
}

// -------------------------------------------------------------------- launchers
template <typename R> static size_t ana_smem(int ty, int tx) {
    const int IH = 2 * ty + MAX_FILTER - 2, IWP = (2 * tx + MAX_FILTER - 2) | 1;
    return (size_t)(IH * IWP + 2 * IH * (tx + 1)) * sizeof(R);
}
template <typename R> static size_t syn_smem(int ty, int tx) {
    const int NKy = ty / 2 + MAX_FILTER / 2, NKx = tx / 2 + MAX_FILTER / 2;
    return (size_t)(4 * NKy * NKx + 2 * ty * (NKx | 1) + ty * (tx + 1)) * sizeof(R);
}

template <typename R>
static cudaError_t analysis(const pd_plan* p, const R* x, R* out, R* ds, const int32_t* active, int mode, R alpha,
                            cudaStream_t s, const R* wt = nullptr) {
    cudaError_t e;
    const int ny = p->g.ny, nx = p->g.nx, b = p->b, L = p->L;
    const R scale = R(1.0 / std::sqrt((double)b));
    const int64_t n = (int64_t)ny * nx;
    int dgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 4);
    if (mode == 0)
        k_dirac<R, 0><<<dgrid, 256, 0, s>>>(x, out, out, nullptr, p->filt_len, active, b, n, scale, alpha);
    else
        k_dirac<R, 1><<<dgrid, 256, 0, s>>>(x, out, ds, wt, p->filt_len, active, b, n, scale, alpha);
    if ((e = cudaGetLastError())) return e;
    if (p->n_wavelet == 0) return cudaSuccess;
    for (int lev = 0; lev < L; ++lev) {
        const int hy = (ny >> lev) / 2, hx = (nx >> lev) / 2;
        const int ty = std::min(AT, hy), tx = std::min(AT, hx);
        dim3 grid((hx + tx - 1) / tx, (hy + ty - 1) / ty, b);
        const R* llin = (const R*)p->ll[(lev + 1) & 1];
        R* llout = (R*)p->ll[lev & 1];
        const size_t sm = ana_smem<R>(ty, tx);
        if ((e = ensure_smem(k_dwt_level<R, 0>, sm)) || (e = ensure_smem(k_dwt_level<R, 1>, sm))) return e;
        if (mode == 0)
            k_dwt_level<R, 0><<<grid, NT_W, sm, s>>>(x, llin, llout, out, nullptr, nullptr, (const R*)p->filt,
                                                     p->filt_len, active, lev, L, ny, nx, scale, alpha);
        else
            k_dwt_level<R, 1><<<grid, NT_W, sm, s>>>(x, llin, llout, out, ds, wt, (const R*)p->filt, p->filt_len,
                                                     active, lev, L, ny, nx, scale, alpha);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

template <typename R>
static cudaError_t synthesis(const pd_plan* p, const R* coef, R* out, const int32_t* active, int mode,
                             cudaStream_t s) {
    cudaError_t e;
    const int ny = p->g.ny, nx = p->g.nx, b = p->b, L = p->L;
    const R scale = R(1.0 / std::sqrt((double)b));
    const int64_t n = (int64_t)ny * nx;
    if (p->n_wavelet > 0) {
        for (int lev = L - 1; lev >= 0; --lev) {
            const int my = ny >> lev, mx = nx >> lev;
            const int ty = std::min(ST, my), tx = std::min(ST, mx);
            dim3 grid((mx + tx - 1) / tx, (my + ty - 1) / ty, b);
            if ((e = ensure_smem(k_idwt_level<R>, syn_smem<R>(ty, tx)))) return e;
            // levels L-1 .. 1 rebuild the approximations, level 0 each basis's full image
            R* dst = lev > 0 ? (R*)p->ll[lev & 1] : (R*)p->synpart;
            const int64_t stride = lev > 0 ? (int64_t)(ny / 2) * (nx / 2) : n;
            k_idwt_level<R><<<grid, NT_W, syn_smem<R>(ty, tx), s>>>(
                coef, (const R*)p->ll[(lev + 1) & 1], dst, (const R*)p->filt, p->filt_len,
                mode == 1 ? active : nullptr, lev, L, ny, nx, stride);
            if ((e = cudaGetLastError())) return e;
        }
    }
    const int ctas = (int)std::min<int64_t>((n / 4 + 255) / 256, (int64_t)p->num_sms * 8);
    if (mode == 0)
        k_syn_sum<R, 0><<<ctas, 256, 0, s>>>(coef, (const R*)p->synpart, p->filt_len, active, b, n, out, scale);
    else
        k_syn_sum<R, 1><<<ctas, 256, 0, s>>>(coef, (const R*)p->synpart, p->filt_len, active, b, n, out, scale);
    return cudaGetLastError();
}

template <typename R>
cudaError_t psi_adj_plain(const pd_plan* p, const R* x, R* coeffs, cudaStream_t s) {
    return analysis<R>(p, x, coeffs, nullptr, p->ones_basis, 0, R(0), s);
}

template <typename R>
cudaError_t psi_plain(const pd_plan* p, const R* coeffs, R* x, cudaStream_t s) {
    return synthesis<R>(p, coeffs, x, p->ones_basis, 0, s);
}

// w = delta / (delta + |w|) in place (the reweighting rule of the weighted analysis prior)
template <typename R>
__global__ void k_sara_rule(R* __restrict__ w, int64_t n, R delta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = delta / (delta + fabs(w[i]));
}

template <typename R>
cudaError_t sara_weights(const pd_plan* p, const R* x, double delta, R* w, cudaStream_t s) {
    cudaError_t e = psi_adj_plain<R>(p, x, w, s);
    if (e) return e;
    const int64_t n = (int64_t)p->b * p->g.ny * p->g.nx;
    const int ctas = (int)std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8);
    k_sara_rule<R><<<ctas, 256, 0, s>>>(w, n, (R)delta);
    return cudaGetLastError();
}

template <typename R>
cudaError_t sparsity_dual(const pd_plan* p, const R* xt, R* s, R* st, const int32_t* basis_active, double alpha,
                          cudaStream_t str, const R* wt) {
    prof_mark(PH_ANALYSIS, 0, str);
    cudaError_t e = analysis<R>(p, xt, s, (R*)p->ds, basis_active, 1, (R)alpha, str, wt);
    prof_mark(PH_ANALYSIS, 1, str);
    if (e) return e;
    prof_mark(PH_SYNTHESIS, 0, str);
    e = synthesis<R>(p, (const R*)p->ds, st, basis_active, 1, str);
    prof_mark(PH_SYNTHESIS, 1, str);
    return e;
}

// -------------------------------------------------------------------- allocation-free analysis
// pd_apply_psi_adj_noalloc runs the same analysis kernels as pd_apply_psi_adj, but
// without a plan: its scratch lives in this file-scope device array instead of memory
// allocated with cudaMalloc. Every GPU that loads the library holds the array until
// exit; every call shares it. Layout: the db1..db8 filter tables in FP64 and FP32
// (written once per device at set-up), then the per-call region: the filter table and
// flags of the call's bases (written by a kernel from its by-value arguments, so a call
// never copies from host memory) and the two approximation buffers of the level loop.
constexpr size_t PSI_STATIC_BYTES = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_psi_static[PSI_STATIC_BYTES];

static size_t align256(size_t n) { return (n + 255) & ~size_t(255); }
constexpr size_t DB_TAB_D = 9 * MAX_FILTER * sizeof(double);   // [9][16], row 0 (Dirac) all zero
constexpr size_t DB_TAB_F = 9 * MAX_FILTER * sizeof(float);
static size_t psi_static_fixed() { return align256(DB_TAB_D) + align256(DB_TAB_F); }

static std::mutex g_psi_static_mu;
static void* g_psi_static_addr[64];       // device address of g_psi_static, per device
static int g_psi_static_sms[64];

// One-time set-up for device `dev` (current): the device address of the static array
// (host code may not use the symbol itself as a pointer), the SM count, and the
// Daubechies tables, written with a synchronous copy before the first call's kernels.
static pd_status psi_static_setup(int dev, void** addr, int* sms) {
    std::lock_guard<std::mutex> lock(g_psi_static_mu);
    if (dev < 0 || dev >= 64) return set_error(PD_ENOTSUP, "pd_apply_psi_adj_noalloc: device index above 63");
    if (!g_psi_static_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_psi_static);
        if (e != cudaSuccess || ptr == nullptr)
            return set_error(PD_ECUDA, "pd_apply_psi_adj_noalloc: cudaGetSymbolAddress of the static scratch failed");
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return set_error(PD_ECUDA, "pd_apply_psi_adj_noalloc: cannot query the SM count");
        std::vector<unsigned char> tab(psi_static_fixed(), 0);
        double* td = (double*)tab.data();
        float* tf = (float*)(tab.data() + align256(DB_TAB_D));
        for (int k = 1; k <= 8; ++k) {
            const std::vector<double> h = daubechies(k);
            for (size_t j = 0; j < h.size(); ++j) { td[k * MAX_FILTER + j] = h[j]; tf[k * MAX_FILTER + j] = (float)h[j]; }
        }
        if (cudaMemcpy(ptr, tab.data(), tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return set_error(PD_ECUDA, "pd_apply_psi_adj_noalloc: writing the filter tables failed");
        g_psi_static_addr[dev] = ptr;
        g_psi_static_sms[dev] = n;
    }
    *addr = g_psi_static_addr[dev];
    *sms = g_psi_static_sms[dev];
    return PD_OK;
}

// The call's bases, passed by value as a kernel argument.
struct BasisList {
    int32_t id[MAX_BASES];
    int32_t b;
};

// Per-call filter table [b][MAX_FILTER], filter lengths and all-active flags of the
// call's bases, from the static db tables.
template <typename R>
__global__ void k_psi_call_tables(BasisList bl, const R* __restrict__ db, R* __restrict__ filt,
                                  int32_t* __restrict__ flen, int32_t* __restrict__ ones) {
    const int i = threadIdx.x;
    if (i >= bl.b * MAX_FILTER) return;
    const int k = i / MAX_FILTER, j = i - k * MAX_FILTER;
    const int id = bl.id[k];
    filt[i] = db[id * MAX_FILTER + j];
    if (j == 0) {
        flen[k] = id == 0 ? 0 : 2 * id;
        ones[k] = 1;
    }
}

template <typename R>
static pd_status psi_adj_static_t(const R* x, R* coeffs, int nx, int ny, int L, const int32_t* ids, int b,
                                  unsigned char* scratch, int sms, cudaStream_t s) {
    const R* db = (const R*)(scratch + (sizeof(R) == 8 ? 0 : align256(DB_TAB_D)));
    unsigned char* call = scratch + psi_static_fixed();
    const size_t filt_bytes = align256((size_t)b * MAX_FILTER * sizeof(R));
    const size_t flag_bytes = align256((size_t)b * sizeof(int32_t));
    const size_t ll_bytes = align256((size_t)b * (ny / 2) * (nx / 2) * sizeof(R));
    R* filt = (R*)call;
    int32_t* flen = (int32_t*)(call + filt_bytes);
    int32_t* ones = (int32_t*)(call + filt_bytes + flag_bytes);
    R* ll[2] = {(R*)(call + filt_bytes + 2 * flag_bytes), (R*)(call + filt_bytes + 2 * flag_bytes + ll_bytes)};
    BasisList bl{};
    bl.b = b;
    int nwav = 0;
    for (int k = 0; k < b; ++k) {
        bl.id[k] = ids[k];
        nwav += ids[k] > 0;
    }
    cudaError_t e;
    k_psi_call_tables<R><<<1, MAX_BASES * MAX_FILTER, 0, s>>>(bl, db, filt, flen, ones);
    if ((e = cudaGetLastError())) return set_error(PD_ECUDA, cudaGetErrorString(e));
    const R scale = R(1.0 / std::sqrt((double)b));
    const int64_t n = (int64_t)ny * nx;
    const int dgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4);
    k_dirac<R, 0><<<dgrid, 256, 0, s>>>(x, coeffs, coeffs, nullptr, flen, ones, b, n, scale, R(0));
    if ((e = cudaGetLastError())) return set_error(PD_ECUDA, cudaGetErrorString(e));
    if (nwav == 0) return PD_OK;
    for (int lev = 0; lev < L; ++lev) {
        const int hy = (ny >> lev) / 2, hx = (nx >> lev) / 2;
        const int ty = std::min(AT, hy), tx = std::min(AT, hx);
        dim3 grid((hx + tx - 1) / tx, (hy + ty - 1) / ty, b);
        const size_t sm = ana_smem<R>(ty, tx);
        if ((e = ensure_smem(k_dwt_level<R, 0>, sm))) return set_error(PD_ECUDA, cudaGetErrorString(e));
        k_dwt_level<R, 0><<<grid, NT_W, sm, s>>>(x, ll[(lev + 1) & 1], ll[lev & 1], coeffs, nullptr, nullptr, filt,
                                                 flen, ones, lev, L, ny, nx, scale, R(0));
        if ((e = cudaGetLastError())) return set_error(PD_ECUDA, cudaGetErrorString(e));
    }
    return PD_OK;
}

}  // namespace pdgb

extern "C" pd_status pd_apply_psi_adj_noalloc(const void* x, void* coeffs, int32_t nx, int32_t ny, int32_t levels,
                                              const int32_t* basis_ids, int32_t nbases, int32_t precision,
                                              void* stream) {
    using namespace pdgb;
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (!x || !coeffs || !basis_ids) return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: null pointer");
    if (!pow2(nx) || !pow2(ny) || nx < 16 || ny < 16 || nx > 8192 || ny > 8192)
        return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: image sides must be powers of two in [16, 8192]");
    // bounded before the shift test (a shift by 32 or more is undefined)
    if (levels < 1 || levels > 13 || (nx >> levels) < 1 || (ny >> levels) < 1)
        return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: levels must satisfy 1 <= L <= 13 and n >> L >= 1");
    if (nbases < 1 || nbases > MAX_BASES) return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: nbases in [1, 16]");
    for (int k = 0; k < nbases; ++k)
        if (basis_ids[k] < 0 || basis_ids[k] > 8)
            return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: basis ids must be 0 (Dirac) or 1..8");
    if (precision != PD_F32 && precision != PD_F64)
        return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: precision must be PD_F32 or PD_F64");
    const size_t rsz = precision == PD_F64 ? 8 : 4;
    const size_t need = psi_static_fixed() + align256((size_t)nbases * MAX_FILTER * rsz) +
                        2 * align256((size_t)nbases * 4) + 2 * align256((size_t)nbases * (ny / 2) * (nx / 2) * rsz);
    if (need > PSI_STATIC_BYTES) {
        static thread_local char msg[160];
        snprintf(msg, sizeof msg,
                 "pd_apply_psi_adj_noalloc: needs %zu bytes of scratch, the static array holds %zu "
                 "(use pd_apply_psi_adj with a plan)", need, PSI_STATIC_BYTES);
        return set_error(PD_EINVAL, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(PD_ECUDA, "pd_apply_psi_adj_noalloc: no current device");
    cudaStream_t s = (cudaStream_t)stream;
    // the array's address is per device: the stream must belong to the current device
    if (s != nullptr) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess)
            return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: cannot query the stream's device");
        if (sdev != dev)
            return set_error(PD_EINVAL, "pd_apply_psi_adj_noalloc: the stream belongs to another device than the current one");
    }
    void* addr = nullptr;
    int sms = 0;
    pd_status st = psi_static_setup(dev, &addr, &sms);
    if (st != PD_OK) return st;
    return precision == PD_F64
               ? psi_adj_static_t<double>((const double*)x, (double*)coeffs, nx, ny, levels, basis_ids, nbases,
                                          (unsigned char*)addr, sms, s)
               : psi_adj_static_t<float>((const float*)x, (float*)coeffs, nx, ny, levels, basis_ids, nbases,
                                         (unsigned char*)addr, sms, s);
}

namespace pdgb {

template cudaError_t psi_adj_plain<float>(const pd_plan*, const float*, float*, cudaStream_t);
template cudaError_t psi_adj_plain<double>(const pd_plan*, const double*, double*, cudaStream_t);
template cudaError_t psi_plain<float>(const pd_plan*, const float*, float*, cudaStream_t);
template cudaError_t psi_plain<double>(const pd_plan*, const double*, double*, cudaStream_t);
template cudaError_t sparsity_dual<float>(const pd_plan*, const float*, float*, float*, const int32_t*, double,
                                          cudaStream_t, const float*);
template cudaError_t sparsity_dual<double>(const pd_plan*, const double*, double*, double*, const int32_t*, double,
                                           cudaStream_t, const double*);
template cudaError_t sara_weights<float>(const pd_plan*, const float*, double, float*, cudaStream_t);
template cudaError_t sara_weights<double>(const pd_plan*, const double*, double, double*, cudaStream_t);

}  // namespace pdgb
