// Sparse interpolation G (degridding) and its adjoint G^T (gridding) with a
// separable J x J Kaiser-Bessel kernel evaluated on the fly (Sec. 2; the paper's
// experiments use 8 x 8 kernels, Sec. 5), fused with the data-fidelity dual
// update of Algorithm 1 step 8 (l2-ball projection, eq. proj-L2) and the
// gridding of the dual change for step 9.
//
// Visibilities are stored in (tile, block) order. A point at continuous grid
// coordinate g has base cell floor(g) (kept mod K as an integer) and fraction
// g - floor(g) (kept in the working precision, computed in FP64 at plan time);
// its taps are the cells floor(g) - J/2 + 1 ... floor(g) + J/2 (mod K), with
// weight phi(fraction + J/2 - 1 - a) for tap a.
//
// Gridding uses ownership instead of global atomics: one CTA per tile
// accumulates its visibilities in shared memory over the tile plus its halo,
// adds the interior to U (nobody else writes it in that launch) and parks the
// halo ring; a second launch adds each tile's neighbours' rings to its border.
#include "common.cuh"
#include "plan.hpp"

namespace pdgb {

template <typename R, int J>
__device__ __forceinline__ void kb_taps(R frac, R* w, R two_over_j, R beta) {
#pragma unroll
    for (int a = 0; a < J; ++a) w[a] = kb_weight<R>(frac + R(J / 2 - 1 - a), two_over_j, beta);
}

template <typename R, int J>
__device__ __forceinline__ cplx_t<R> interp(const cplx_t<R>* __restrict__ grid, int cell, R fx, R fy, int Kx, int Ky,
                                            R two_over_j, R beta) {
    using C2 = cplx_t<R>;
    R wx[J], wy[J];
    kb_taps<R, J>(fx, wx, two_over_j, beta);
    kb_taps<R, J>(fy, wy, two_over_j, beta);
    const int bx = cell & 0xFFFF, by = cell >> 16;
    C2 acc = mk<C2>(R(0), R(0));
#pragma unroll
    for (int b = 0; b < J; ++b) {
        const int ky = (by - J / 2 + 1 + b) & (Ky - 1);
        C2 rs = mk<C2>(R(0), R(0));
#pragma unroll
        for (int a = 0; a < J; ++a) {
            const int kx = (bx - J / 2 + 1 + a) & (Kx - 1);
            const C2 gv = __ldg(&grid[panel_off(ky, kx, Ky)]);
            rs.x += wx[a] * gv.x;
            rs.y += wx[a] * gv.y;
        }
        acc.x += wy[b] * rs.x;
        acc.y += wy[b] * rs.y;
    }
    return acc;
}

// ---------------------------------------------------------------- degridding
// plain: out_user[perm[m]] = (G grid)_m over all chunks
template <typename R, int J>
__global__ void __launch_bounds__(256) k_degrid_plain(const cplx_t<R>* __restrict__ grid, cplx_t<R>* __restrict__ out,
                                                      const int32_t* __restrict__ cell, const R* __restrict__ fxs,
                                                      const R* __restrict__ fys, const int32_t* __restrict__ perm,
                                                      const int32_t* __restrict__ cstart, const int32_t* __restrict__ cend,
                                                      int nchunk, int Kx, int Ky, R two_over_j, R beta) {
    for (int w = blockIdx.x; w < nchunk; w += gridDim.x) {
        const int e = cend[w];
        for (int m = cstart[w] + threadIdx.x; m < e; m += blockDim.x)
            out[perm[m]] = interp<R, J>(grid, cell[m], fxs[m], fys[m], Kx, Ky, two_over_j, beta);
    }
}

// pd: r = v + G b - y for the listed chunks (all of active blocks); FP64 partial
// sums of ||r||^2 and ||G b - y||^2 per chunk.
template <typename R, int J>
__global__ void __launch_bounds__(256) k_degrid_dual(const cplx_t<R>* __restrict__ grid, const cplx_t<R>* __restrict__ y,
                                                     const cplx_t<R>* __restrict__ v, cplx_t<R>* __restrict__ rbuf,
                                                     const int32_t* __restrict__ cell, const R* __restrict__ fxs,
                                                     const R* __restrict__ fys, const int32_t* __restrict__ cstart,
                                                     const int32_t* __restrict__ cend, const int32_t* __restrict__ list,
                                                     const int32_t* __restrict__ count, double* __restrict__ part,
                                                     int Kx, int Ky, R two_over_j, R beta) {
    using C2 = cplx_t<R>;
    __shared__ double red[32];
    const int n = *count;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int c = list[w];
        const int e = cend[c];
        double ar = 0.0, ad = 0.0;
        for (int m = cstart[c] + threadIdx.x; m < e; m += blockDim.x) {
            const C2 gb = interp<R, J>(grid, cell[m], fxs[m], fys[m], Kx, Ky, two_over_j, beta);
            const C2 yy = y[m], vv = v[m];
            const C2 d = csub(gb, yy);
            const C2 r = cadd(vv, d);
            rbuf[m] = r;
            ar += (double)r.x * r.x + (double)r.y * r.y;
            ad += (double)d.x * d.x + (double)d.y * d.y;
        }
        const double sr = block_sum(ar, red);
        const double sd = block_sum(ad, red);
        if (threadIdx.x == 0) { part[2 * c] = sr; part[2 * c + 1] = sd; }
    }
}

// Per-block FP64 norms in a fixed order, the ball scale c_i = max(0, 1 - eps_i/||r_i||)
// of step 8 (so v_new = c_i r_i = z - P_B(z)), and the residual norm for Sec. 4.
template <typename R>
__global__ void k_block_norms(const double* __restrict__ part, const int32_t* __restrict__ bcs,
                              const int32_t* __restrict__ active, const double* __restrict__ eps,
                              double* __restrict__ bnorm, R* __restrict__ scale, double* __restrict__ res_norm, int d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d || !active[i]) return;
    double sr = 0.0, sd = 0.0;
    for (int c = bcs[i]; c < bcs[i + 1]; ++c) { sr += part[2 * c]; sd += part[2 * c + 1]; }
    bnorm[2 * i] = sr;
    bnorm[2 * i + 1] = sd;
    const double nr = sqrt(sr);
    const double sc = nr > eps[i] ? 1.0 - eps[i] / nr : 0.0;
    scale[i] = (R)sc;
    res_norm[i] = sqrt(sd);
}

// ---------------------------------------------------------------- gridding
__device__ __forceinline__ int ring_index(int ey, int ex, const Geo& g) {
    const int H = g.halo_lo, A = g.halo_hi, E = g.ext, T = g.tile;
    if (ey < H) return ey * E + ex;
    if (ey >= H + T) return (H + ey - H - T) * E + ex;
    const int base = (H + A) * E;
    if (ex < H) return base + (ey - H) * H + ex;
    return base + T * H + (ey - H) * A + (ex - H - T);
}

// mode 0 (plain): d = y_user[perm[m]] for every visibility, U interior overwritten.
// mode 1 (pd): for active blocks v_new = scale_i r, d = v_new - v_old, v <- v_new, U interior += .
template <typename R, int J, int MODE>
__global__ void __launch_bounds__(256) k_grid(const cplx_t<R>* __restrict__ src, const cplx_t<R>* __restrict__ rbuf,
                                              cplx_t<R>* __restrict__ v, const R* __restrict__ scale,
                                              const int32_t* __restrict__ active, const int32_t* __restrict__ cell,
                                              const R* __restrict__ fxs, const R* __restrict__ fys,
                                              const int32_t* __restrict__ perm, const int32_t* __restrict__ seg_start,
                                              const int32_t* __restrict__ seg_block,
                                              const int32_t* __restrict__ tile_seg_start,
                                              const int32_t* __restrict__ list, const int32_t* __restrict__ count,
                                              cplx_t<R>* __restrict__ U, cplx_t<R>* __restrict__ ring, Geo g,
                                              R two_over_j, R beta) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    R* acc = reinterpret_cast<R*>(smraw);   // [ext*ext] re then [ext*ext] im
    const int E = g.ext, EE = E * E;
    const int n = *count;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int t = list[w];
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int y0 = ty * g.tile, x0 = tx * g.tile;
        for (int i = threadIdx.x; i < 2 * EE; i += blockDim.x) acc[i] = R(0);
        __syncthreads();
        for (int sg = tile_seg_start[t]; sg < tile_seg_start[t + 1]; ++sg) {
            if (MODE == 1 && !active[seg_block[sg]]) continue;
            const R sc = MODE == 1 ? scale[seg_block[sg]] : R(0);
            const int e = seg_start[sg + 1];
            for (int m = seg_start[sg] + threadIdx.x; m < e; m += blockDim.x) {
                C2 dv;
                if (MODE == 0) {
                    dv = src[perm[m]];
                } else {
                    const C2 r = rbuf[m], vo = v[m];
                    const C2 vn = cscale(r, sc);
                    v[m] = vn;
                    dv = csub(vn, vo);
                }
                R wx[J], wy[J];
                kb_taps<R, J>(fxs[m], wx, two_over_j, beta);
                kb_taps<R, J>(fys[m], wy, two_over_j, beta);
                const int c = cell[m];
                const int ex0 = (c & 0xFFFF) - x0, ey0 = (c >> 16) - y0;
#pragma unroll
                for (int b = 0; b < J; ++b) {
                    const R wr = wy[b] * dv.x, wi = wy[b] * dv.y;
                    R* rowp = acc + (ey0 + b) * E + ex0;
#pragma unroll
                    for (int a = 0; a < J; ++a) {
                        atomicAdd(rowp + a, wx[a] * wr);
                        atomicAdd(rowp + a + EE, wx[a] * wi);
                    }
                }
            }
        }
        __syncthreads();
        const int H = g.halo_lo, T = g.tile;
        for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
            const int iy = i / T, ix = i - iy * T;
            const int k = (iy + H) * E + ix + H;
            const int64_t off = panel_off(y0 + iy, x0 + ix, g.Ky);
            C2 val = mk<C2>(acc[k], acc[k + EE]);
            if (MODE == 1) val = cadd(U[off], val);
            U[off] = val;
        }
        C2* rg = ring + (int64_t)t * g.ring;
        for (int i = threadIdx.x; i < EE; i += blockDim.x) {
            const int ey = i / E, ex = i - ey * E;
            if (ey >= H && ey < H + T && ex >= H && ex < H + T) continue;
            rg[ring_index(ey, ex, g)] = mk<C2>(acc[i], acc[i + EE]);
        }
        __syncthreads();
    }
}

// Add the neighbours' halo rings to each tile's border cells (periodic grid).
template <typename R>
__global__ void __launch_bounds__(256) k_halo_merge(cplx_t<R>* __restrict__ U, const cplx_t<R>* __restrict__ ring,
                                                    const int32_t* __restrict__ flag, Geo g) {
    using C2 = cplx_t<R>;
    const int H = g.halo_lo, A = g.halo_hi, T = g.tile, E = g.ext;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        int nb[9];
        bool any = false;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int dy = k / 3 - 1, dx = k % 3 - 1;
            const int nty = (ty + dy + g.nty) % g.nty, ntx = (tx + dx + g.ntx) % g.ntx;
            nb[k] = nty * g.ntx + ntx;
            if (k != 4 && flag[nb[k]]) any = true;
        }
        if (!any) continue;
        for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
            const int iy = i / T, ix = i - iy * T;
            if (iy >= A && iy < T - H && ix >= A && ix < T - H) continue;
            C2 sum = mk<C2>(R(0), R(0));
            bool hit = false;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (k == 4) continue;
                const int dy = k / 3 - 1, dx = k % 3 - 1;
                const int ey = iy - dy * T + H, ex = ix - dx * T + H;
                if (ey < 0 || ey >= E || ex < 0 || ex >= E) continue;
                if (!flag[nb[k]]) continue;
                sum = cadd(sum, ring[(int64_t)nb[k] * g.ring + ring_index(ey, ex, g)]);
                hit = true;
            }
            if (hit) {
                const int64_t off = panel_off(ty * T + iy, tx * T + ix, g.Ky);
                U[off] = cadd(U[off], sum);
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
template <typename R> static int grid_ctas(const pd_plan* p, int work) {
    int c = p->num_sms * 8;
    return work < c ? (work > 0 ? work : 1) : c;
}

#define PD_J_DISPATCH(J_, CALL)           \
    switch (J_) {                         \
        case 2: { constexpr int JJ = 2; CALL; } break;   \
        case 4: { constexpr int JJ = 4; CALL; } break;   \
        case 6: { constexpr int JJ = 6; CALL; } break;   \
        case 8: { constexpr int JJ = 8; CALL; } break;   \
        case 10: { constexpr int JJ = 10; CALL; } break; \
        case 12: { constexpr int JJ = 12; CALL; } break; \
        case 14: { constexpr int JJ = 14; CALL; } break; \
        case 16: { constexpr int JJ = 16; CALL; } break; \
        default: return cudaErrorInvalidValue;           \
    }

template <typename R>
cudaError_t degrid_plain(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out_user, cudaStream_t s) {
    const Geo& g = p->g;
    const R toj = R(2.0 / g.J), beta = R(g.beta);
    const int ctas = (int)std::min<int64_t>(p->nchunk, (int64_t)p->num_sms * 8);
    PD_J_DISPATCH(g.J, (k_degrid_plain<R, JJ><<<ctas, 256, 0, s>>>(
        grid, out_user, p->cell, (const R*)p->fx, (const R*)p->fy, p->perm, p->chunk_start, p->chunk_end,
        (int)p->nchunk, g.Kx, g.Ky, toj, beta)));
    return cudaGetLastError();
}

template <typename R>
cudaError_t degrid_dual(const pd_plan* p, const cplx_t<R>* grid, const DualArgs& a, const int32_t* chunks,
                        const int32_t* counts, cudaStream_t s) {
    const Geo& g = p->g;
    const R toj = R(2.0 / g.J), beta = R(g.beta);
    const int ctas = (int)std::min<int64_t>(p->nchunk, (int64_t)p->num_sms * 8);
    prof_mark(PH_DEGRID, 0, s);
    PD_J_DISPATCH(g.J, (k_degrid_dual<R, JJ><<<ctas, 256, 0, s>>>(
        grid, (const cplx_t<R>*)a.y, (const cplx_t<R>*)a.v, (cplx_t<R>*)p->rbuf, p->cell, (const R*)p->fx,
        (const R*)p->fy, p->chunk_start, p->chunk_end, chunks, counts, p->chunk_part, g.Kx, g.Ky, toj, beta)));
    prof_mark(PH_DEGRID, 1, s);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    prof_mark(PH_NORMS, 0, s);
    k_block_norms<R><<<(p->d + 127) / 128, 128, 0, s>>>(p->chunk_part, p->block_chunk_start, a.block_active, a.eps,
                                                       p->blk_norm, (R*)p->blk_scale, a.res_norm, p->d);
    prof_mark(PH_NORMS, 1, s);
    return cudaGetLastError();
}

template <typename R, int J, int MODE> static cudaError_t grid_attr(size_t smem) {
    return ensure_smem(k_grid<R, J, MODE>, smem);
}

template <typename R>
static cudaError_t launch_grid(const pd_plan* p, int mode, const cplx_t<R>* src, const DualArgs* a,
                               const int32_t* tiles, const int32_t* counts, const int32_t* flags, cplx_t<R>* U,
                               cudaStream_t s) {
    const Geo& g = p->g;
    const R toj = R(2.0 / g.J), beta = R(g.beta);
    const size_t smem = (size_t)2 * g.ext * g.ext * sizeof(R);
    const int ctas = std::min(g.ntiles, p->num_sms * 4);
    cudaError_t e = cudaSuccess;
    prof_mark(PH_GRID, 0, s);
    if (mode == 0) {
        PD_J_DISPATCH(g.J, (e = grid_attr<R, JJ, 0>(smem),
                            e ? (void)0 : (void)(k_grid<R, JJ, 0><<<ctas, 256, smem, s>>>(
                                src, nullptr, nullptr, nullptr, nullptr, p->cell, (const R*)p->fx, (const R*)p->fy,
                                p->perm, p->seg_start, p->seg_block, p->tile_seg_start, tiles, counts, U,
                                (cplx_t<R>*)p->ringbuf, g, toj, beta))));
    } else {
        PD_J_DISPATCH(g.J, (e = grid_attr<R, JJ, 1>(smem),
                            e ? (void)0 : (void)(k_grid<R, JJ, 1><<<ctas, 256, smem, s>>>(
                                nullptr, (const cplx_t<R>*)p->rbuf, (cplx_t<R>*)a->v, (const R*)p->blk_scale,
                                a->block_active, p->cell, (const R*)p->fx, (const R*)p->fy, p->perm, p->seg_start,
                                p->seg_block, p->tile_seg_start, tiles, counts, U, (cplx_t<R>*)p->ringbuf, g, toj,
                                beta))));
    }
    prof_mark(PH_GRID, 1, s);
    if (e) return e;
    if ((e = cudaGetLastError())) return e;
    prof_mark(PH_HALO, 0, s);
    k_halo_merge<R><<<std::min(g.ntiles, p->num_sms * 8), 256, 0, s>>>(U, (const cplx_t<R>*)p->ringbuf, flags, g);
    prof_mark(PH_HALO, 1, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t grid_plain(const pd_plan* p, const cplx_t<R>* y_user, cplx_t<R>* U, cudaStream_t s) {
    return launch_grid<R>(p, 0, y_user, nullptr, p->all_tiles, p->counts_all + 1, p->tile_ones, U, s);
}

template <typename R>
cudaError_t grid_dual(const pd_plan* p, const DualArgs& a, const int32_t* tiles, const int32_t* counts,
                      const int32_t* tile_active, cplx_t<R>* U, cudaStream_t s) {
    return launch_grid<R>(p, 1, nullptr, &a, tiles, counts + 1, tile_active, U, s);
}

template cudaError_t degrid_plain<float>(const pd_plan*, const float2*, float2*, cudaStream_t);
template cudaError_t degrid_plain<double>(const pd_plan*, const double2*, double2*, cudaStream_t);
template cudaError_t degrid_dual<float>(const pd_plan*, const float2*, const DualArgs&, const int32_t*,
                                        const int32_t*, cudaStream_t);
template cudaError_t degrid_dual<double>(const pd_plan*, const double2*, const DualArgs&, const int32_t*,
                                         const int32_t*, cudaStream_t);
template cudaError_t grid_plain<float>(const pd_plan*, const float2*, float2*, cudaStream_t);
template cudaError_t grid_plain<double>(const pd_plan*, const double2*, double2*, cudaStream_t);
template cudaError_t grid_dual<float>(const pd_plan*, const DualArgs&, const int32_t*, const int32_t*,
                                      const int32_t*, float2*, cudaStream_t);
template cudaError_t grid_dual<double>(const pd_plan*, const DualArgs&, const int32_t*, const int32_t*,
                                       const int32_t*, double2*, cudaStream_t);

}  // namespace pdgb
