// The interpolation G held as a sparse matrix (Sec. 2: G has J^2 non-zero entries per
// row, the kernel footprint of each visibility; Sec. 3 splits it into the blocks G_i).
// The plan stores it once, on the device, in CSR form with a fixed row length: row m
// (a visibility, internal order) owns the entries m J^2 ... m J^2 + J^2 - 1, so the row
// pointer is m J^2 and is not stored. Entry b J + a is the footprint cell of row tap b
// and column tap a: its column index packs the grid cell as (ky << 16 | kx) and its
// value is phi_y(b) phi_x(a), evaluated in FP64 at plan time and rounded once to the
// working precision.
//
// Both products keep the tile structure of the on-the-fly kernels (visibilities sorted
// by tile, the tile's window of the grid in shared memory, four colour launches for the
// gridding), but take every column and weight from the stored matrix:
// * degridding: eight lanes per visibility, lane b walks footprint row b (two 16-byte
//   loads of columns and two of weights in FP32), gathers from the staged window and
//   the eight row sums are added by a fixed shuffle tree;
// * gridding: one warp per visibility at a time, lane l adds entries 2l and 2l + 1 into
//   the warp's private copy of the window (the J^2 cells of one footprint are distinct,
//   so no atomics), the warps' copies are summed in warp order into U. Deterministic.
#include <algorithm>
#include <type_traits>

#include "gridding.cuh"

namespace pdgb {

// ---------------------------------------------------------------- building G
// Row m of G: the J^2 (cell, weight) entries of visibility m.
template <typename R, int J>
__global__ void k_build_csr(const int32_t* __restrict__ cell, const R* __restrict__ fxs, const R* __restrict__ fys,
                            int64_t M, Geo g, int32_t* __restrict__ col, R* __restrict__ val) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double wx[J], wy[J];
    const double toj = 2.0 / g.J;
#pragma unroll
    for (int a = 0; a < J; ++a) {
        wx[a] = kb_weight<double>((double)fxs[m] + (J / 2 - 1 - a), toj, g.beta);
        wy[a] = kb_weight<double>((double)fys[m] + (J / 2 - 1 - a), toj, g.beta);
    }
    const int c = cell[m], by = c >> 16, bx = c & 0xFFFF;
    int32_t* cp = col + m * (J * J);
    R* vp = val + m * (J * J);
#pragma unroll
    for (int b = 0; b < J; ++b) {
        const int ky = (by - g.halo_lo + b) & (g.Ky - 1);
#pragma unroll
        for (int a = 0; a < J; ++a) {
            cp[b * J + a] = (ky << 16) | ((bx - g.halo_lo + a) & (g.Kx - 1));
            vp[b * J + a] = (R)(wy[b] * wx[a]);
        }
    }
}

// Row m of the DDE-aware G (Sec. 2): the JK x JK interpolation kernel convolved with the
// point's d x d Fourier-domain DDE kernel D_m (offsets -h .. h), a footprint of
// g.J = JK + d - 1 cells per axis starting g.halo_lo = JK/2 - 1 + h cells before the base
// cell. Entry (b', a') = sum over b + i = b', a + j = a' of phi_y(b) phi_x(a) D_m[i][j],
// summed in FP64 and rounded once.
template <typename R, int JK>
__global__ void k_build_csr_dde(const int32_t* __restrict__ cell, const R* __restrict__ fxs,
                                const R* __restrict__ fys, const double2* __restrict__ dde, int dw, int64_t M,
                                Geo g, double beta, int32_t* __restrict__ col, cplx_t<R>* __restrict__ val) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double wx[JK], wy[JK];
    const double toj = 2.0 / JK;
#pragma unroll
    for (int a = 0; a < JK; ++a) {
        wx[a] = kb_weight<double>((double)fxs[m] + (JK / 2 - 1 - a), toj, beta);
        wy[a] = kb_weight<double>((double)fys[m] + (JK / 2 - 1 - a), toj, beta);
    }
    const int c = cell[m], by = c >> 16, bx = c & 0xFFFF;
    const int Jf = g.J;
    const double2* D = dde + m * dw * dw;
    int32_t* cp = col + m * Jf * Jf;
    cplx_t<R>* vp = val + m * Jf * Jf;
    for (int bq = 0; bq < Jf; ++bq) {
        const int ky = (by - g.halo_lo + bq) & (g.Ky - 1);
        for (int aq = 0; aq < Jf; ++aq) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < dw; ++i) {
                const int b = bq - i;
                if (b < 0 || b >= JK) continue;
                for (int j = 0; j < dw; ++j) {
                    const int a = aq - j;
                    if (a < 0 || a >= JK) continue;
                    const double w = wy[b] * wx[a];
                    re += w * D[i * dw + j].x;
                    im += w * D[i * dw + j].y;
                }
            }
            cp[bq * Jf + aq] = (ky << 16) | ((bx - g.halo_lo + aq) & (g.Kx - 1));
            vp[bq * Jf + aq] = mk<cplx_t<R>>((R)re, (R)im);
        }
    }
}

cudaError_t build_csr(pd_plan* p, cudaStream_t s) {
    const Geo& g = p->g;
    const int64_t M = p->M;
    const unsigned nb = (unsigned)((M + 127) / 128);
    if (M == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (p->csr_cplx) {
        if (p->kb_J != 2 && p->kb_J != 4 && p->kb_J != 6) return cudaErrorInvalidValue;   // J + d - 1 <= 8, d >= 3
        // the DDE kernels go to the device once, for this build only
        double2* dd = nullptr;
        const size_t bytes = p->h_dde.size() * sizeof(double);
        if ((e = cudaMalloc(&dd, bytes))) return e;
        if ((e = cudaMemcpy(dd, p->h_dde.data(), bytes, cudaMemcpyHostToDevice))) { cudaFree(dd); return e; }
        if (p->prec == PD_F64) {
            PD_J_DISPATCH(p->kb_J, (k_build_csr_dde<double, JJ><<<nb, 128, 0, s>>>(
                                       p->cell, (const double*)p->fx, (const double*)p->fy, dd, p->dde, M, g,
                                       g.beta, p->csr_col, (double2*)p->csr_val)));
        } else {
            PD_J_DISPATCH(p->kb_J, (k_build_csr_dde<float, JJ><<<nb, 128, 0, s>>>(
                                       p->cell, (const float*)p->fx, (const float*)p->fy, dd, p->dde, M, g,
                                       g.beta, p->csr_col, (float2*)p->csr_val)));
        }
        if (!e) e = cudaGetLastError();
        const cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(dd);
        return e ? e : e2;
    }
    if (p->prec == PD_F64) {
        PD_J_DISPATCH(g.J, (k_build_csr<double, JJ><<<nb, 128, 0, s>>>(p->cell, (const double*)p->fx,
                                                                       (const double*)p->fy, M, g, p->csr_col,
                                                                       (double*)p->csr_val)));
    } else {
        PD_J_DISPATCH(g.J, (k_build_csr<float, JJ><<<nb, 128, 0, s>>>(p->cell, (const float*)p->fx,
                                                                      (const float*)p->fy, M, g, p->csr_col,
                                                                      (float*)p->csr_val)));
    }
    return e ? e : cudaGetLastError();
}

// Weight arithmetic for real rows (interpolation only) and complex rows (DDE-aware G):
// wmac: s += w g; wmacc: a += conj(w) v (the adjoint's weight).
__device__ __forceinline__ void wmac(float w, float2 g, float& sx, float& sy) { sx += w * g.x; sy += w * g.y; }
__device__ __forceinline__ void wmac(double w, double2 g, double& sx, double& sy) { sx += w * g.x; sy += w * g.y; }
__device__ __forceinline__ void wmac(float2 w, float2 g, float& sx, float& sy) {
    sx += w.x * g.x - w.y * g.y;
    sy += w.x * g.y + w.y * g.x;
}
__device__ __forceinline__ void wmac(double2 w, double2 g, double& sx, double& sy) {
    sx += w.x * g.x - w.y * g.y;
    sy += w.x * g.y + w.y * g.x;
}
__device__ __forceinline__ void wmacc(float w, float vr, float vi, float2& a) { a.x += w * vr; a.y += w * vi; }
__device__ __forceinline__ void wmacc(double w, double vr, double vi, double2& a) { a.x += w * vr; a.y += w * vi; }
__device__ __forceinline__ void wmacc(float2 w, float vr, float vi, float2& a) {
    a.x += w.x * vr + w.y * vi;
    a.y += w.x * vi - w.y * vr;
}
__device__ __forceinline__ void wmacc(double2 w, double vr, double vi, double2& a) {
    a.x += w.x * vr + w.y * vi;
    a.y += w.x * vi - w.y * vr;
}

// J consecutive entries of one footprint row (16-byte loads where the row is 16-byte aligned)
template <typename W, int J>
__device__ __forceinline__ void load_row(const int32_t* __restrict__ cp, const W* __restrict__ vp, int* cc, W* ww) {
    if constexpr (J == 8 && std::is_same<W, float>::value) {
        const int4 c0 = *reinterpret_cast<const int4*>(cp), c1 = *reinterpret_cast<const int4*>(cp + 4);
        const float4 v0 = *reinterpret_cast<const float4*>(vp), v1 = *reinterpret_cast<const float4*>(vp + 4);
        cc[0] = c0.x; cc[1] = c0.y; cc[2] = c0.z; cc[3] = c0.w; cc[4] = c1.x; cc[5] = c1.y; cc[6] = c1.z; cc[7] = c1.w;
        ww[0] = v0.x; ww[1] = v0.y; ww[2] = v0.z; ww[3] = v0.w; ww[4] = v1.x; ww[5] = v1.y; ww[6] = v1.z; ww[7] = v1.w;
    } else if constexpr (J == 8 && std::is_same<W, float2>::value) {
        const int4 c0 = *reinterpret_cast<const int4*>(cp), c1 = *reinterpret_cast<const int4*>(cp + 4);
        cc[0] = c0.x; cc[1] = c0.y; cc[2] = c0.z; cc[3] = c0.w; cc[4] = c1.x; cc[5] = c1.y; cc[6] = c1.z; cc[7] = c1.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(vp + 2 * q);
            ww[2 * q] = make_float2(v.x, v.y);
            ww[2 * q + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int a = 0; a < J; ++a) { cc[a] = cp[a]; ww[a] = vp[a]; }
    }
}

// ---------------------------------------------------------------- degridding
// MODE 0: out_user[perm[m]] = (G grid)_m; MODE 1: r = v + G b - y for visibilities of
// active blocks with the FP64 per-segment sums of ||r||^2 and ||G b - y||^2 (the outputs
// of the on-the-fly degridding, same work items and tile claiming).
template <typename R, typename W, int J, int MODE>
__global__ void __launch_bounds__(256) k_degrid_csr(
    const cplx_t<R>* __restrict__ grid, cplx_t<R>* __restrict__ out, const cplx_t<R>* __restrict__ y,
    const cplx_t<R>* __restrict__ v, cplx_t<R>* __restrict__ rbuf, const int32_t* __restrict__ col,
    const W* __restrict__ val, const int32_t* __restrict__ perm, const int32_t* __restrict__ seg_start,
    const int32_t* __restrict__ seg_block, const int32_t* __restrict__ tile_seg_start,
    const int32_t* __restrict__ active, const int32_t* __restrict__ list, const int32_t* __restrict__ count,
    double* __restrict__ seg_part, int max_segs, Geo g, int* __restrict__ next_tile, int batch, int64_t gstride,
    int64_t ostride) {
    using C2 = cplx_t<R>;
    constexpr int GL = 8;   // lanes per visibility, lane b of a group on footprint row b (b < J)
    extern __shared__ __align__(16) unsigned char smraw[];
    const int E = g.ext, H = g.halo_lo;
    C2* win = reinterpret_cast<C2*>(smraw);                              // [E][E]
    double* part = reinterpret_cast<double*>(win + E * E + (E * E & 1)); // [8 warps][max_segs][2]
    int* act_seg = reinterpret_cast<int*>(part + 16 * max_segs);
    int* act_pre = act_seg + max_segs;
    __shared__ int nact_s, tile_s;
    const int warp = threadIdx.x >> 5, grp = threadIdx.x / GL, b = threadIdx.x % GL;
    const int ngrp = blockDim.x / GL;
    const int n = *count;
    for (;;) {
        if (threadIdx.x == 0) tile_s = atomicAdd(next_tile, 1);
        __syncthreads();
        const int w = tile_s;
        if (w >= n * batch) break;
        const int t = list[w / batch], img = w % batch;
        const C2* gimg = grid + (int64_t)img * gstride;
        C2* oimg = MODE == 0 ? out + (int64_t)img * ostride : out;
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int wy0 = ty * g.tile - H, wx0 = tx * g.tile - H;     // window origin (unwrapped)
        const int seg0 = tile_seg_start[t], nseg_t = tile_seg_start[t + 1] - seg0;
        list_active_segments(seg0, nseg_t, seg_block, MODE == 1 ? active : nullptr, seg_start, act_seg, act_pre,
                             &nact_s);
        for (int i = threadIdx.x; i < E * E; i += blockDim.x) {
            const int ey = i / E, ex = i - ey * E;
            win[i] = half_grid_at(gimg, (wy0 + ey) & (g.Ky - 1), (wx0 + ex) & (g.Kx - 1), g);
        }
        if (MODE == 1)
            for (int i = threadIdx.x; i < 16 * nseg_t; i += blockDim.x) part[i] = 0.0;
        __syncthreads();
        const int nact = nact_s, total = act_pre[nact];
        double* mypart = part + 2 * nseg_t * warp;
        int j = 0;
        for (int base = 0; base < total; base += ngrp) {
            const int pos = base + grp;
            const bool ok = pos < total;
            int m = 0;
            R sx = 0, sy = 0;
            if (ok) {
                while (act_pre[j + 1] <= pos) ++j;
                m = seg_start[act_seg[j]] + pos - act_pre[j];
                if (b < J) {
                    int cc[J];
                    W ww[J];
                    load_row<W, J>(col + (int64_t)m * (J * J) + b * J, val + (int64_t)m * (J * J) + b * J, cc, ww);
#pragma unroll
                    for (int a = 0; a < J; ++a) {
                        const int ey = ((cc[a] >> 16) - wy0) & (g.Ky - 1), ex = ((cc[a] & 0xFFFF) - wx0) & (g.Kx - 1);
                        wmac(ww[a], win[ey * E + ex], sx, sy);
                    }
                }
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            const bool lead = ok && b == 0;
            R ar = R(0), ad = R(0);
            if (lead) {
                if (MODE == 0) {
                    oimg[perm[m]] = mk<C2>(sx, sy);
                } else {
                    const C2 yy = y[m], vv = v[m];
                    const R dx = sx - yy.x, dy = sy - yy.y;
                    const C2 r = mk<C2>(vv.x + dx, vv.y + dy);
                    rbuf[m] = r;
                    ar = r.x * r.x + r.y * r.y;
                    ad = dx * dx + dy * dy;
                }
            }
            if (MODE == 1) warp_seg_add(lead, j, ar, ad, mypart);
        }
        __syncthreads();
        if (MODE == 1) {
            for (int k = threadIdx.x; k < nact; k += blockDim.x) {
                double sr = 0.0, sd = 0.0;
                for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) {
                    sr += part[2 * nseg_t * wp + 2 * k];
                    sd += part[2 * nseg_t * wp + 2 * k + 1];
                }
                seg_part[2 * act_seg[k]] = sr;
                seg_part[2 * act_seg[k] + 1] = sd;
            }
        }
        __syncthreads();
    }
}

template <typename R, typename W, int J, int MODE>
static cudaError_t degrid_csr_w(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out, const DualArgs* a,
                                const int32_t* tiles, const int32_t* count, int ctas, cudaStream_t s, int batch) {
    const Geo& g = p->g;
    const int ms = std::max(p->max_tile_segs, 1);
    const size_t win = (size_t)g.ext * g.ext + (g.ext * g.ext & 1);
    const size_t smem = win * sizeof(cplx_t<R>) + (size_t)16 * ms * sizeof(double) + (size_t)(2 * ms + 1) * sizeof(int);
    cudaError_t e = ensure_smem(k_degrid_csr<R, W, J, MODE>, smem);
    if (e) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid_csr<R, W, J, MODE>, 256, smem) ==
            cudaSuccess && per_sm > 0)
        ctas = std::min(ctas, per_sm * p->num_sms);
    if ((e = cudaMemsetAsync(p->sched + 4, 0, sizeof(int32_t), s))) return e;
    k_degrid_csr<R, W, J, MODE><<<ctas, 256, smem, s>>>(
        grid, out, a ? (const cplx_t<R>*)a->y : nullptr, a ? (const cplx_t<R>*)a->v : nullptr,
        (cplx_t<R>*)p->rbuf, p->csr_col, (const W*)p->csr_val, p->perm, p->seg_start, p->seg_block,
        p->tile_seg_start, a ? a->block_active : nullptr, tiles, count, p->seg_part, ms, g, p->sched + 4, batch,
        (int64_t)(g.nx / 4 + 1) * 4 * g.Ky, (int64_t)p->M);
    return cudaGetLastError();
}

template <typename R, int J, int MODE>
cudaError_t launch_degrid_csr(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out, const DualArgs* a,
                              const int32_t* tiles, const int32_t* count, int ctas, cudaStream_t s, int batch) {
    return p->csr_cplx ? degrid_csr_w<R, cplx_t<R>, J, MODE>(p, grid, out, a, tiles, count, ctas, s, batch)
                       : degrid_csr_w<R, R, J, MODE>(p, grid, out, a, tiles, count, ctas, s, batch);
}

// ---------------------------------------------------------------- gridding
template <typename R> __device__ __forceinline__ void ld2(const R* p, R& a, R& b) {
    if constexpr (sizeof(R) == 4) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        a = q.x; b = q.y;
    } else {
        const double2 q = *reinterpret_cast<const double2*>(p);
        a = q.x; b = q.y;
    }
}

__device__ __forceinline__ void ld2(const float2* p, float2& a, float2& b) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    a = make_float2(q.x, q.y); b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld2(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }

// The raw inputs of one visibility to grid: MODE 1 r, v_old and the block's ball scale;
// MODE 0 the input value (in a).
template <typename R> struct GridRaw {
    cplx_t<R> a, b;
    R sc;
    int m;
};

template <typename R, int MODE>
__device__ __forceinline__ void grid_raw(GridRaw<R>& in, int pos, int& j, const int* act_seg, const int* act_pre,
                                         const int32_t* __restrict__ seg_start, const int32_t* __restrict__ seg_block,
                                         const cplx_t<R>* __restrict__ src, const cplx_t<R>* __restrict__ rbuf,
                                         const cplx_t<R>* __restrict__ v, const int32_t* __restrict__ perm,
                                         const R* __restrict__ scale) {
    while (act_pre[j + 1] <= pos) ++j;
    const int sg = act_seg[j];
    const int m = seg_start[sg] + pos - act_pre[j];
    in.m = m;
    if (MODE == 1) {
        in.a = rbuf[m];
        in.b = v[m];
        in.sc = scale[seg_block[sg]];
    } else {
        in.a = src[perm[m]];
    }
}

// MODE 1: v_new = c_i r (step 8) is written and v_new - v_old returned; MODE 0: the input
template <typename R, int MODE>
__device__ __forceinline__ cplx_t<R> grid_raw_value(const GridRaw<R>& in, cplx_t<R>* __restrict__ v) {
    if (MODE == 0) return in.a;
    const cplx_t<R> vn = cscale(in.a, in.sc);
    v[in.m] = vn;
    return csub(vn, in.b);
}

// Each warp takes a contiguous share of the tile's active visibilities (fixed by the
// warp index, so the summation order is too) and adds them one at a time into its own
// E x E window; the windows are then summed in warp order and added to U.
template <typename R, typename W, int J, int MODE>
__global__ void __launch_bounds__(256, 2) k_grid_csr(
    const cplx_t<R>* __restrict__ src, const cplx_t<R>* __restrict__ rbuf, cplx_t<R>* __restrict__ v,
    const R* __restrict__ scale, const int32_t* __restrict__ active, const int32_t* __restrict__ col,
    const W* __restrict__ val, const int32_t* __restrict__ perm, const int32_t* __restrict__ seg_start,
    const int32_t* __restrict__ seg_block, const int32_t* __restrict__ tile_seg_start,
    const int32_t* __restrict__ list, const int32_t* __restrict__ count, cplx_t<R>* __restrict__ U, int max_segs,
    Geo g, int* __restrict__ next_tile, int batch, int64_t sstride, int64_t ustride) {
    using C2 = cplx_t<R>;
    constexpr int NE = J * J;                 // entries per row of G (<= 64: two per lane)
    constexpr int PB = 8;                     // visibilities whose entries are loaded together
    extern __shared__ __align__(16) unsigned char smraw[];
    const int E = g.ext, EE = E * E, H = g.halo_lo;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2* wins = reinterpret_cast<C2*>(smraw);                 // [nw][E][E]
    int* act_seg = reinterpret_cast<int*>(wins + (size_t)nw * EE);
    int* act_pre = act_seg + max_segs;
    __shared__ int nact_s, tile_s;
    C2* win = wins + (size_t)warp * EE;
    const int n = *count;
    const int e0 = 2 * lane;
    const bool has = e0 < NE;                 // J^2 is even: entries e0, e0 + 1 together
    for (;;) {
        if (threadIdx.x == 0) tile_s = atomicAdd(next_tile, 1);
        __syncthreads();
        const int w = tile_s;
        if (w >= n * batch) break;
        const int t = list[w / batch], img = w % batch;
        const C2* simg = MODE == 0 ? src + (int64_t)img * sstride : src;
        C2* uimg = U + (int64_t)img * ustride;
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int oy = ty * g.tile, ox = tx * g.tile;
        const int wy0 = oy - H, wx0 = ox - H;
        const int seg0 = tile_seg_start[t], nseg_t = tile_seg_start[t + 1] - seg0;
        list_active_segments(seg0, nseg_t, seg_block, MODE == 1 ? active : nullptr, seg_start, act_seg, act_pre,
                             &nact_s);
        for (int i = threadIdx.x; i < nw * EE; i += blockDim.x) wins[i] = mk<C2>(R(0), R(0));
        __syncthreads();
        const int total = act_pre[nact_s];
        const int p0 = (int)((int64_t)total * warp / nw), p1 = (int)((int64_t)total * (warp + 1) / nw);
        int j = 0;
        // the raw inputs of the next 32 visibilities are loaded one chunk ahead
        GridRaw<R> nx{};
        if (p0 + lane < p1) grid_raw<R, MODE>(nx, p0 + lane, j, act_seg, act_pre, seg_start, seg_block, simg, rbuf, v, perm, scale);
        for (int q0 = p0; q0 < p1; q0 += 32) {
            // lane q: visibility q0 + q and its value to grid (MODE 1 also writes v_new)
            const GridRaw<R> cur = nx;
            const int nq = min(32, p1 - q0);
            C2 dv = mk<C2>(R(0), R(0));
            if (lane < nq) dv = grid_raw_value<R, MODE>(cur, v);
            if (q0 + 32 + lane < p1)
                grid_raw<R, MODE>(nx, q0 + 32 + lane, j, act_seg, act_pre, seg_start, seg_block, simg, rbuf, v, perm, scale);
            for (int qb = 0; qb < nq; qb += PB) {
                int2 cc[PB];
                W w0[PB], w1[PB];
#pragma unroll
                for (int k = 0; k < PB; ++k) {
                    const int mq = __shfl_sync(0xffffffffu, cur.m, (qb + k) & 31);
                    cc[k] = make_int2(0, 0);
                    w0[k] = w1[k] = W{};
                    if (has && qb + k < nq) {
                        const int64_t o = (int64_t)mq * NE + e0;
                        cc[k] = *reinterpret_cast<const int2*>(col + o);
                        ld2(val + o, w0[k], w1[k]);   // entries e0, e0 + 1 (16-byte aligned pair)
                    }
                }
#pragma unroll
                for (int k = 0; k < PB; ++k) {
                    const R vr = __shfl_sync(0xffffffffu, dv.x, (qb + k) & 31);
                    const R vi = __shfl_sync(0xffffffffu, dv.y, (qb + k) & 31);
                    if (has && qb + k < nq) {
                        const int i0 = (((cc[k].x >> 16) - wy0) & (g.Ky - 1)) * E + (((cc[k].x & 0xFFFF) - wx0) & (g.Kx - 1));
                        const int i1 = (((cc[k].y >> 16) - wy0) & (g.Ky - 1)) * E + (((cc[k].y & 0xFFFF) - wx0) & (g.Kx - 1));
                        C2 a0 = win[i0];
                        wmacc(w0[k], vr, vi, a0);
                        win[i0] = a0;
                        C2 a1 = win[i1];
                        wmacc(w1[k], vr, vi, a1);
                        win[i1] = a1;
                    }
                    __syncwarp();     // the next visibility's lanes may read these cells
                }
            }
        }
        __syncthreads();
        add_window<R>(uimg, oy, ox, g, [&](int ey, int ex) {
            C2 sum = wins[ey * E + ex];
            for (int k = 1; k < nw; ++k) sum = cadd(sum, wins[(size_t)k * EE + ey * E + ex]);
            return sum;
        });
        __syncthreads();
    }
}

template <typename R, typename W, int J, int MODE>
static cudaError_t grid_csr_w(const pd_plan* p, const cplx_t<R>* src, const DualArgs* a, const int32_t* tiles,
                              const int32_t* count, cplx_t<R>* U, int* next_tile, cudaStream_t s, int batch) {
    const Geo& g = p->g;
    const int ms = std::max(p->max_tile_segs, 1);
    const size_t winb = (size_t)g.ext * g.ext * sizeof(cplx_t<R>);
    // eight warps unless their windows do not fit (large tiles in FP64)
    const int nw = (int)std::max<size_t>(1, std::min<size_t>(8, ((size_t)200 << 10) / winb));
    const size_t smem = nw * winb + (size_t)(2 * ms + 1) * sizeof(int);
    cudaError_t e = ensure_smem(k_grid_csr<R, W, J, MODE>, smem);
    if (e) return e;
    int per_sm = 0, ctas = std::min(g.ntiles * batch, p->num_sms * 8);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_csr<R, W, J, MODE>, nw * 32, smem) ==
            cudaSuccess && per_sm > 0)
        ctas = std::min(ctas, per_sm * p->num_sms);
    k_grid_csr<R, W, J, MODE><<<ctas, nw * 32, smem, s>>>(
        src, (const cplx_t<R>*)p->rbuf, a ? (cplx_t<R>*)a->v : nullptr, (const R*)p->blk_scale,
        a ? a->block_active : nullptr, p->csr_col, (const W*)p->csr_val, p->perm, p->seg_start, p->seg_block,
        p->tile_seg_start, tiles, count, U, ms, g, next_tile, batch, (int64_t)p->M, (int64_t)g.Kx * g.Ky);
    return cudaGetLastError();
}

template <typename R, int J, int MODE>
cudaError_t launch_grid_csr(const pd_plan* p, const cplx_t<R>* src, const DualArgs* a, const int32_t* tiles,
                            const int32_t* count, cplx_t<R>* U, int* next_tile, cudaStream_t s, int batch) {
    return p->csr_cplx ? grid_csr_w<R, cplx_t<R>, J, MODE>(p, src, a, tiles, count, U, next_tile, s, batch)
                       : grid_csr_w<R, R, J, MODE>(p, src, a, tiles, count, U, next_tile, s, batch);
}

#define PD_CSR_INST(R_, J_)                                                                                      \
    template cudaError_t launch_degrid_csr<R_, J_, 0>(const pd_plan*, const cplx_t<R_>*, cplx_t<R_>*,            \
                                                      const DualArgs*, const int32_t*, const int32_t*, int,      \
                                                      cudaStream_t, int);                                        \
    template cudaError_t launch_degrid_csr<R_, J_, 1>(const pd_plan*, const cplx_t<R_>*, cplx_t<R_>*,            \
                                                      const DualArgs*, const int32_t*, const int32_t*, int,      \
                                                      cudaStream_t, int);                                        \
    template cudaError_t launch_grid_csr<R_, J_, 0>(const pd_plan*, const cplx_t<R_>*, const DualArgs*,          \
                                                    const int32_t*, const int32_t*, cplx_t<R_>*, int*,           \
                                                    cudaStream_t, int);                                          \
    template cudaError_t launch_grid_csr<R_, J_, 1>(const pd_plan*, const cplx_t<R_>*, const DualArgs*,          \
                                                    const int32_t*, const int32_t*, cplx_t<R_>*, int*,           \
                                                    cudaStream_t, int);
PD_CSR_INST(float, 2)
PD_CSR_INST(float, 4)
PD_CSR_INST(float, 6)
PD_CSR_INST(float, 8)
PD_CSR_INST(double, 2)
PD_CSR_INST(double, 4)
PD_CSR_INST(double, 6)
PD_CSR_INST(double, 8)

}  // namespace pdgb
