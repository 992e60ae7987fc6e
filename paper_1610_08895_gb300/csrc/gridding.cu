// Sparse interpolation G (degridding) and its adjoint G^T (gridding) with a
// separable J x J Kaiser-Bessel kernel evaluated on the fly (Sec. 2; the paper's
// experiments use 8 x 8 kernels, Sec. 5), fused with the data-fidelity dual
// update of Algorithm 1 step 8 (l2-ball projection, eq. proj-L2) and the
// gridding of the dual change for step 9.
//
// Visibilities are stored in (tile, block, super-cell, row, column) order of
// their base cell: each (tile, block) pair is a contiguous segment. Per tile, the
// segments of active blocks are listed in shared memory and worked on as one
// concatenated range, so inactive blocks cost nothing and batches stay full. A point at continuous grid coordinate g has base cell floor(g) (kept
// mod K) and fraction g - floor(g) (working precision, computed in FP64 at plan
// time); its taps are the cells floor(g) - J/2 + 1 ... floor(g) + J/2 (mod K),
// with weight phi(fraction + J/2 - 1 - a) for tap a.
//
// Both directions work tile by tile (one CTA owns a T x T tile at a time) on the
// tile plus a halo of J/2 - 1 cells before and J/2 after:
// * degridding stages that window of F Z x (held as its half grid: the columns
//   kx <= nx, the others by conjugate symmetry) in shared memory and gathers from it;
// * gridding accumulates the window in shared memory and adds the whole window
//   (tile and halo) to U. The tiles are gridded in four launches, one per tile colour
//   (tile row and column parity): the windows of two tiles of one colour are disjoint,
//   so no two CTAs of a launch touch the same cell of U. No global atomics.
#include <algorithm>

#include "gridding.cuh"

namespace pdgb {

// ---------------------------------------------------------------- degridding
// The global inputs of one point to degrid (MODE 1 also its y and v).
template <typename R> struct DegridIn {
    cplx_t<R> yy, vv;
    R fx, fy;
    int c, m;
};

template <typename R, int MODE>
__device__ __forceinline__ void degrid_load(DegridIn<R>& in, int pos, int& j, const int* act_seg, const int* act_pre,
                                            const int32_t* __restrict__ seg_start, const int32_t* __restrict__ cell,
                                            const R* __restrict__ fxs, const R* __restrict__ fys,
                                            const cplx_t<R>* __restrict__ y, const cplx_t<R>* __restrict__ v) {
    while (act_pre[j + 1] <= pos) ++j;
    const int m = seg_start[act_seg[j]] + pos - act_pre[j];
    in.m = m;
    in.c = cell[m];
    in.fx = fxs[m];
    in.fy = fys[m];
    if (MODE == 1) {
        in.yy = y[m];
        in.vv = v[m];
    }
}

// MODE 0 (plain): out_user[perm[m]] = (G grid)_m for every visibility of the listed tiles.
// MODE 1 (pd): for visibilities of active blocks r = v + G b - y, with FP64 sums of
// ||r||^2 and ||G b - y||^2 per (tile, block) segment (per-warp slots, summed in warp order).
template <typename R, int J, int MODE>
__global__ void __launch_bounds__(256, J <= 8 ? (sizeof(R) == 4 ? 5 : 3) : 1) k_degrid(const cplx_t<R>* __restrict__ grid, cplx_t<R>* __restrict__ out,
                                                const cplx_t<R>* __restrict__ y, const cplx_t<R>* __restrict__ v,
                                                cplx_t<R>* __restrict__ rbuf, const int32_t* __restrict__ cell,
                                                const R* __restrict__ fxs, const R* __restrict__ fys,
                                                const int32_t* __restrict__ perm,
                                                const int32_t* __restrict__ seg_start,
                                                const int32_t* __restrict__ seg_block,
                                                const int32_t* __restrict__ tile_seg_start,
                                                const int32_t* __restrict__ active, const int32_t* __restrict__ list,
                                                const int32_t* __restrict__ count, double* __restrict__ seg_part,
                                                int max_segs, Geo g, R two_over_j, R beta, const KbPoly kp,
                                                int* __restrict__ next_tile, int batch, int64_t gstride,
                                                int64_t ostride) {
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    // FP32: the window twice, row stride EP (even), the second copy shifted left by one
    // column, so every footprint row is J/2 aligned 16-byte pairs in one of the copies.
    // FP64: one copy, row stride E.
    constexpr bool PAIRS = sizeof(R) == 4;
    const int EP = PAIRS ? ((g.ext + 2) & ~1) : g.ext;
    C2* win = reinterpret_cast<C2*>(smraw);                              // [ext][EP] (x2 in FP32)
    double* part = reinterpret_cast<double*>(win + (PAIRS ? 2 : 1) * g.ext * EP);  // [8 warps][max_segs][2]
    int* act_seg = reinterpret_cast<int*>(part + 16 * max_segs);        // [max_segs]
    int* act_pre = act_seg + max_segs;                                   // [max_segs + 1]
    __shared__ int nact_s, tile_s;
    const int E = g.ext, T = g.tile, H = g.halo_lo;
    const int warp = threadIdx.x >> 5;
    const int n = *count;
    for (;;) {
        // tiles are taken from the heaviest-first list one at a time by whichever CTA is free
        if (threadIdx.x == 0) tile_s = atomicAdd(next_tile, 1);
        __syncthreads();
        const int w = tile_s;
        if (w >= n * batch) break;
        // work item w: tile w / batch of the list for image w mod batch (a batch of plain
        // applications; the heaviest tiles of every image come first)
        const int t = list[w / batch], img = w % batch;
        const cplx_t<R>* gimg = grid + (int64_t)img * gstride;
        cplx_t<R>* oimg = MODE == 0 ? out + (int64_t)img * ostride : out;
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int oy = ty * T, ox = tx * T;
        const int seg0 = tile_seg_start[t], nseg_t = tile_seg_start[t + 1] - seg0;
        list_active_segments(seg0, nseg_t, seg_block, MODE == 1 ? active : nullptr, seg_start, act_seg, act_pre,
                             &nact_s);
        for (int i = threadIdx.x; i < E * E; i += blockDim.x) {
            const int ey = i / E, ex = i - ey * E;
            const C2 gv = half_grid_at(gimg, (oy - H + ey) & (g.Ky - 1), (ox - H + ex) & (g.Kx - 1), g);
            win[ey * EP + ex] = gv;
            if (PAIRS && ex > 0) win[E * EP + ey * EP + ex - 1] = gv;
        }
        if (MODE == 1)
            for (int i = threadIdx.x; i < 16 * nseg_t; i += blockDim.x) part[i] = 0.0;
        __syncthreads();
        const int nact = nact_s, total = act_pre[nact];
        double* mypart = part + 2 * nseg_t * warp;
        int j = 0;   // segment cursor: positions only grow, so it only moves forward
        // the inputs of the point blockDim.x positions ahead are loaded while this one is worked on
        DegridIn<R> nx{};
        if ((int)threadIdx.x < total) degrid_load<R, MODE>(nx, threadIdx.x, j, act_seg, act_pre, seg_start, cell, fxs, fys, y, v);
        for (int base = 0; base < total; base += blockDim.x) {
            const int pos = base + threadIdx.x;
            const bool ok = pos < total;
            const DegridIn<R> in = nx;
            const int jcur = j;
            if (pos + (int)blockDim.x < total)
                degrid_load<R, MODE>(nx, pos + blockDim.x, j, act_seg, act_pre, seg_start, cell, fxs, fys, y, v);
            R ar = R(0), ad = R(0);     // squares in the working precision (exact for FP64)
            if (ok) {
                const int m = in.m;
                R wx[J], wy[J];
                kb_taps<R, J>(in.fx, wx, two_over_j, beta, kp);
                kb_taps<R, J>(in.fy, wy, two_over_j, beta, kp);
                const int c = in.c;
                const int r0 = (c >> 16) - oy, c0 = (c & 0xFFFF) - ox;   // footprint origin in the window
                R sx = 0, sy = 0;
                if constexpr (PAIRS) {
                    const float4* bp = reinterpret_cast<const float4*>(
                        (c0 & 1) ? win + E * EP + r0 * EP + c0 - 1 : win + r0 * EP + c0);
#pragma unroll
                    for (int b = 0; b < J; ++b) {
                        R rx = 0, ry = 0;
#pragma unroll
                        for (int a = 0; a < J / 2; ++a) {
                            const float4 q = bp[(b * EP >> 1) + a];
                            rx += wx[2 * a] * q.x + wx[2 * a + 1] * q.z;
                            ry += wx[2 * a] * q.y + wx[2 * a + 1] * q.w;
                        }
                        sx += wy[b] * rx;
                        sy += wy[b] * ry;
                    }
                } else {
                    const C2* bp = win + r0 * EP + c0;
#pragma unroll
                    for (int b = 0; b < J; ++b) {
                        R rx = 0, ry = 0;
#pragma unroll
                        for (int a = 0; a < J; ++a) {
                            const C2 gv = bp[b * EP + a];
                            rx += wx[a] * gv.x;
                            ry += wx[a] * gv.y;
                        }
                        sx += wy[b] * rx;
                        sy += wy[b] * ry;
                    }
                }
                if (MODE == 0) {
                    oimg[perm[m]] = mk<C2>(sx, sy);
                } else {
                    const R dx = sx - in.yy.x, dy = sy - in.yy.y;
                    const C2 r = mk<C2>(in.vv.x + dx, in.vv.y + dy);
                    rbuf[m] = r;
                    ar = r.x * r.x + r.y * r.y;
                    ad = dx * dx + dy * dy;
                }
            }
            if (MODE == 1) warp_seg_add(ok, jcur, ar, ad, mypart);
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

// Per-block FP64 norms summed over the block's segments in a fixed order (one warp per
// block: lane-strided partial sums, then a fixed shuffle tree), the ball scale
// c_i = max(0, 1 - eps_i/||r_i||) of step 8 (so v_new = c_i r_i = z - P_B(z)), and the
// residual norm ||G_i b - y_i|| for the adaptive probabilities of Sec. 4.
// norm_only (active == nullptr: every block): only the residual norm is written.
template <typename R>
__global__ void k_block_norms(const double* __restrict__ part, const int32_t* __restrict__ bss,
                              const int32_t* __restrict__ bsl, const int32_t* __restrict__ active,
                              const double* __restrict__ eps, double* __restrict__ bnorm, R* __restrict__ scale,
                              double* __restrict__ res_norm, int d, int norm_only) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= d || (active && !active[i])) return;     // whole warps leave together
    double sr = 0.0, sd = 0.0;
    for (int k = bss[i] + lane; k < bss[i + 1]; k += 32) {
        const int sg = bsl[k];
        sr += part[2 * sg];
        sd += part[2 * sg + 1];
    }
    sr = warp_sum(sr);
    sd = warp_sum(sd);
    if (lane != 0) return;
    if (norm_only) {
        res_norm[i] = sqrt(sd);
        return;
    }
    bnorm[2 * i] = sr;
    bnorm[2 * i + 1] = sd;
    const double nr = sqrt(sr);
    const double sc = nr > eps[i] ? 1.0 - eps[i] / nr : 0.0;
    scale[i] = (R)sc;
    res_norm[i] = sqrt(sd);
}

// ---------------------------------------------------------------- gridding
// Generic J: one thread per visibility, shared-memory atomics per tap.
template <typename R, int J, int MODE>
__global__ void __launch_bounds__(256) k_grid(const cplx_t<R>* __restrict__ src, const cplx_t<R>* __restrict__ rbuf,
                                              cplx_t<R>* __restrict__ v, const R* __restrict__ scale,
                                              const int32_t* __restrict__ active, const int32_t* __restrict__ cell,
                                              const R* __restrict__ fxs, const R* __restrict__ fys,
                                              const int32_t* __restrict__ perm, const int32_t* __restrict__ seg_start,
                                              const int32_t* __restrict__ seg_block,
                                              const int32_t* __restrict__ tile_seg_start,
                                              const int32_t* __restrict__ list, const int32_t* __restrict__ count,
                                              cplx_t<R>* __restrict__ U, int max_segs,
                                              Geo g, R two_over_j, R beta, const KbPoly kp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    R* acc = reinterpret_cast<R*>(smraw);   // [ext*ext] re then [ext*ext] im
    int* act_seg = reinterpret_cast<int*>(acc + 2 * g.ext * g.ext);
    int* act_pre = act_seg + max_segs;
    __shared__ int nact_s;
    const int E = g.ext, EE = E * E;
    const int n = *count;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int t = list[w];
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int oy = ty * g.tile, ox = tx * g.tile;
        const int seg0 = tile_seg_start[t], nseg_t = tile_seg_start[t + 1] - seg0;
        list_active_segments(seg0, nseg_t, seg_block, MODE == 1 ? active : nullptr, seg_start, act_seg, act_pre,
                             &nact_s);
        for (int i = threadIdx.x; i < 2 * EE; i += blockDim.x) acc[i] = R(0);
        __syncthreads();
        const int total = act_pre[nact_s];
        int j = 0;
        for (int pos = threadIdx.x; pos < total; pos += blockDim.x) {
            while (act_pre[j + 1] <= pos) ++j;
            const int sg = act_seg[j];
            const int m = seg_start[sg] + pos - act_pre[j];
            const cplx_t<R> dv = grid_value<R, MODE>(m, src, rbuf, v, perm, MODE == 1 ? scale[seg_block[sg]] : R(0));
            R wx[J], wy[J];
            kb_taps<R, J>(fxs[m], wx, two_over_j, beta, kp);
            kb_taps<R, J>(fys[m], wy, two_over_j, beta, kp);
            const int c = cell[m];
            R* rowp = acc + ((c >> 16) - oy) * E + ((c & 0xFFFF) - ox);
#pragma unroll
            for (int b = 0; b < J; ++b) {
                const R wr = wy[b] * dv.x, wi = wy[b] * dv.y;
#pragma unroll
                for (int a = 0; a < J; ++a) {
                    atomicAdd(rowp + b * E + a, wx[a] * wr);
                    atomicAdd(rowp + b * E + a + EE, wx[a] * wi);
                }
            }
        }
        __syncthreads();
        add_window<R>(U, oy, ox, g, [&](int ey, int ex) { return mk<cplx_t<R>>(acc[ey * E + ex], acc[ey * E + ex + EE]); });
        __syncthreads();
    }
}

// J <= 8 without atomics inside a tile. Warp w of the CTA takes the 8 x 8 super-cells of
// column w of the tile (T/8 warps), so its points' footprints cover the window columns
// 8w .. 8w + 15 only: each warp accumulates into a private window of T + 7 rows and 16
// columns, and the CTA sums the (at most two) windows that cover each cell at the end of
// the tile. Cells are split into 64 classes by (window row mod 8, window column mod 8);
// lane l owns classes (l / 4, 2 (l % 4) + {0, 1}). A J x J footprint (J <= 8) holds at
// most one cell of each class, so the lanes of a warp never touch the same cell. The
// points of a super-cell arrive sorted by base row: over one base row (a "super-row") a
// class has one footprint row and two candidate columns (c and c + 8 of the warp's
// window), and the lane keeps one running sum per candidate cell in registers, adding
// them to its window when the row changes.
// Staging (one lane per point, 32 points per chunk) writes per-class records that make
// the lane's work a fixed-address read: for row class r the weight times the value,
// phi_y(tap) d; for column class c the weight of its tap, negated when the class cell is
// the high candidate (the weights are positive, so the sign carries the choice and the
// lane splits it with max(w, 0) and max(-w, 0)). The staging lane rotates its taps into
// class order in registers (three conditional shifts), so the column record is two
// aligned 16-byte stores and one 8-byte read per lane and point.
constexpr int GW_MAXW = 16;    // warps per CTA: one per super-cell column (tile <= 128)
constexpr int GW_RREC = 9;     // row records per staged point (8, padded against bank conflicts)
constexpr int GW_CREC = 12;    // column record reals per staged point (8, padded: 16-byte rows, no conflicts)
constexpr int GW_WP = 18;      // window pitch (complex): the 16 columns of one super-cell column's footprints,
                               // padded so that the 8 rows a warp's flush touches start in distinct banks

template <typename R> __device__ __forceinline__ void ld2r(const R* p, R& a, R& b) {
    if constexpr (sizeof(R) == 4) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        a = q.x; b = q.y;
    } else {
        const double2 q = *reinterpret_cast<const double2*>(p);
        a = q.x; b = q.y;
    }
}
template <typename R> __device__ __forceinline__ void st4(R* p, R a, R b, R c, R d) {
    if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
        *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
    }
}
// lo, hi += the class weight's low / high part times ry
template <typename C2, typename R> __device__ __forceinline__ void acc_cand(C2& lo, C2& hi, R w, C2 ry) {
    const R wl = w > R(0) ? w : R(0), wh = w < R(0) ? -w : R(0);
    lo.x += wl * ry.x; lo.y += wl * ry.y;
    hi.x += wh * ry.x; hi.y += wh * ry.y;
}

// p[0] += a, p[1] += b (two adjacent complex cells, 16-byte aligned in FP32)
template <typename C2> __device__ __forceinline__ void add2(C2* p, C2 a, C2 b) {
    if constexpr (sizeof(C2) == 8) {
        float4* q = reinterpret_cast<float4*>(p);
        float4 t = *q;
        t.x += a.x; t.y += a.y; t.z += b.x; t.w += b.y;
        *q = t;
    } else {
        p[0] = cadd(p[0], a);
        p[1] = cadd(p[1], b);
    }
}

// Shared memory of one CTA of nw warps (ms: most segments of a tile).
template <typename R>
__host__ __device__ constexpr size_t grid8w_smem(int T, int nw, int ms) {
    return (size_t)nw * (T + 7) * GW_WP * 2 * sizeof(R)                       // windows
           + (size_t)nw * 32 * (GW_RREC * 2 + GW_CREC) * sizeof(R)           // records
           + (size_t)nw * (ms * (T / 8 > 0 ? T / 8 : 1) + 1) * sizeof(R)      // range scales
           + (size_t)nw * (2 * (ms * (T / 8 > 0 ? T / 8 : 1)) + 1) * sizeof(int)   // range starts, prefixes
           + (size_t)(2 * ms + 1) * sizeof(int);                              // active segment lists
}

// The raw inputs of one staged point, loaded a chunk ahead.
template <typename R> struct GridIn {
    cplx_t<R> a, b;     // MODE 1: r and v_old; MODE 0: the input value (a)
    R fx, fy, sc;
    int c, m;
};

template <typename R, int MODE>
__device__ __forceinline__ void grid_load(GridIn<R>& in, int pos, int& j, const int* rpre, const int* rstart,
                                          const R* rscale, const cplx_t<R>* __restrict__ src,
                                          const cplx_t<R>* __restrict__ rbuf, const cplx_t<R>* __restrict__ v,
                                          const int32_t* __restrict__ cell, const R* __restrict__ fxs,
                                          const R* __restrict__ fys, const int32_t* __restrict__ perm) {
    while (rpre[j + 1] <= pos) ++j;
    const int m = rstart[j] + pos - rpre[j];
    in.m = m;
    in.fx = fxs[m];
    in.fy = fys[m];
    in.c = cell[m];
    if (MODE == 1) {
        in.a = rbuf[m];
        in.b = v[m];
        in.sc = rscale[j];
    } else {
        in.a = src[perm[m]];
    }
}

template <typename R, int J, int MODE>
__global__ void __launch_bounds__(GW_MAXW * 32) k_grid8w(
    const cplx_t<R>* __restrict__ src, const cplx_t<R>* __restrict__ rbuf, cplx_t<R>* __restrict__ v,
    const R* __restrict__ scale, const int32_t* __restrict__ active, const int32_t* __restrict__ cell,
    const R* __restrict__ fxs, const R* __restrict__ fys, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ seg_start, const int32_t* __restrict__ seg_block,
    const int32_t* __restrict__ tile_seg_start, const int32_t* __restrict__ sc_start,
    const int32_t* __restrict__ list, const int32_t* __restrict__ count, cplx_t<R>* __restrict__ U, int max_segs,
    Geo g, R two_over_j, R beta, const KbPoly kp, int* __restrict__ next_tile, int batch, int64_t istride,
    int64_t ustride) {
    static_assert(J <= 8 && J % 2 == 0, "class ownership needs J <= 8");
    using C2 = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int T = g.tile, E = g.ext, WR = T + 7, WS = WR * GW_WP;
    const int nsd = T / 8 > 0 ? T / 8 : 1, nsc = nsd * nsd;    // super-cells per side, per tile
    const int nw = blockDim.x >> 5;                             // = nsd
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rcap = max_segs * nsd;                            // ranges a warp can hold
    C2* wins = reinterpret_cast<C2*>(smraw);                    // [nw][WR][GW_WP]
    C2* win = wins + (size_t)warp * WS;
    C2* rrec = wins + (size_t)nw * WS + (size_t)warp * 32 * GW_RREC;
    R* crec = reinterpret_cast<R*>(wins + (size_t)nw * WS + (size_t)nw * 32 * GW_RREC) + (size_t)warp * 32 * GW_CREC;
    R* rscale = reinterpret_cast<R*>(wins + (size_t)nw * WS + (size_t)nw * 32 * GW_RREC) + (size_t)nw * 32 * GW_CREC +
                (size_t)warp * (rcap + 1);
    int* ints = reinterpret_cast<int*>(reinterpret_cast<R*>(wins + (size_t)nw * WS + (size_t)nw * 32 * GW_RREC) +
                                       (size_t)nw * 32 * GW_CREC + (size_t)nw * (rcap + 1));
    int* rstart = ints + warp * (2 * rcap + 1);
    int* rpre = rstart + rcap;                                  // [rcap + 1]
    int* act_seg = ints + nw * (2 * rcap + 1);
    int* act_pre = act_seg + max_segs;
    __shared__ int nact_s, tile_s;
    const int lcy = lane >> 2, lcx = (lane & 3) * 2;
    const int n = *count;
    for (;;) {
        // tiles are taken from the heaviest-first list one at a time by whichever CTA is free
        if (threadIdx.x == 0) tile_s = atomicAdd(next_tile, 1);
        __syncthreads();
        const int w = tile_s;
        if (w >= n * batch) break;
        // work item w: tile w / batch of the list for image w mod batch (plain gridding of a batch)
        const int t = list[w / batch], img = w % batch;
        const cplx_t<R>* simg = MODE == 0 ? src + (int64_t)img * istride : src;
        cplx_t<R>* Uimg = U + (int64_t)img * ustride;
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const int oy = ty * T, ox = tx * T;
        const int seg0 = tile_seg_start[t], nseg_t = tile_seg_start[t + 1] - seg0;
        list_active_segments(seg0, nseg_t, seg_block, MODE == 1 ? active : nullptr, seg_start, act_seg, act_pre,
                             &nact_s);
        for (int i = lane; i < WS; i += 32) win[i] = mk<C2>(R(0), R(0));
        __syncthreads();
        // this warp's ranges: the super-cells of column `warp` of every active segment
        const int nact = nact_s, nr = nact * nsd;
        if (lane == 0) rpre[0] = 0;
        for (int base = 0; base < nr; base += 32) {
            const int k = base + lane;
            int len = 0, st0 = 0;
            R scv = R(0);
            if (k < nr) {
                const int jj = k / nsd, srow = k - jj * nsd;
                const int sg = act_seg[jj];
                const int sc = srow * nsd + warp;
                st0 = sc_start[(int64_t)sg * (nsc + 1) + sc];
                len = sc_start[(int64_t)sg * (nsc + 1) + sc + 1] - st0;
                if (MODE == 1) scv = scale[seg_block[sg]];
            }
            int incl = len;
            for (int o = 1; o < 32; o <<= 1) {
                const int yv = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += yv;
            }
            const int before = base > 0 ? rpre[base] : 0;
            __syncwarp();
            if (k < nr) {
                rstart[k] = st0;
                rscale[k] = scv;
                rpre[k + 1] = before + incl;
            }
            __syncwarp();
        }
        const int total = nr > 0 ? rpre[nr] : 0;
        // chunks of 32 consecutive points of the warp's ranges
        const int nchunk = (total + 31) >> 5;
        int j = 0;            // this lane's range cursor (its positions only grow)
        GridIn<R> in{};
        if (nchunk > 0 && lane < total)
            grid_load<R, MODE>(in, lane, j, rpre, rstart, rscale, simg, rbuf, v, cell, fxs, fys, perm);
        for (int chunk = 0; chunk < nchunk; ++chunk) {
            const int fill = min(32, total - chunk * 32);
            int mykey = -1;   // footprint row of this lane's staged point
            if (lane < fill) {
                C2 d;
                if (MODE == 1) {
                    const C2 vn = cscale(in.a, in.sc);       // step 8: v_new = c_i r
                    v[in.m] = vn;
                    d = csub(vn, in.b);
                } else {
                    d = in.a;
                }
                R wx[J], wy[J];
                kb_taps<R, J>(in.fx, wx, two_over_j, beta, kp);
                kb_taps<R, J>(in.fy, wy, two_over_j, beta, kp);
                const int r0 = (in.c >> 16) - oy, c0 = (in.c & 0xFFFF) - ox;   // footprint origin in the window
                C2* rr = rrec + lane * GW_RREC;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const R wv = b < J ? wy[b] : R(0);
                    rr[(r0 + b) & 7] = mk<C2>(wv * d.x, wv * d.y);
                }
                // class c = (gam + a) mod 8 takes tap a = (c - gam) mod 8; its cell is the high
                // candidate (window column c + 8) when gam + a >= 8, i.e. when c < gam
                const int gam = c0 & 7;                             // c0 = 8 warp + gam
                R cw[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) cw[a] = a < J ? wx[a] : R(0);
#pragma unroll
                for (int sh = 1; sh < 8; sh <<= 1) {
                    const bool on = (gam & sh) != 0;
                    R t[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) t[c] = on ? cw[(c - sh) & 7] : cw[c];
#pragma unroll
                    for (int c = 0; c < 8; ++c) cw[c] = t[c];
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) cw[c] = c < gam ? -cw[c] : cw[c];
                R* cr = crec + lane * GW_CREC;
                st4(cr, cw[0], cw[1], cw[2], cw[3]);
                st4(cr + 4, cw[4], cw[5], cw[6], cw[7]);
                mykey = r0;
            }
            // the next chunk's loads go out now and land while this one is accumulated
            const int nxt = (chunk + 1) * 32 + lane;
            if (nxt < total)
                grid_load<R, MODE>(in, nxt, j, rpre, rstart, rscale, simg, rbuf, v, cell, fxs, fys, perm);
            __syncwarp();
            // runs of consecutive points with the same footprint row: one set of running sums
            // per run, added to the window at its end
            const int prevk = __shfl_up_sync(0xffffffffu, mykey, 1);
            unsigned starts = __ballot_sync(0xffffffffu, lane < fill && (lane == 0 || mykey != prevk));
            while (starts) {
                const int q0 = __ffs(starts) - 1;
                starts &= starts - 1;
                const int q1 = starts ? __ffs(starts) - 1 : fill;
                const int r0 = __shfl_sync(0xffffffffu, mykey, q0);
                // the run's first point starts the running sums, the others add to them two at a time
                C2 lo0 = mk<C2>(R(0), R(0)), hi0 = lo0, lo1 = lo0, hi1 = lo0;
                int q = q0;
                for (; q + 1 < q1; q += 2) {
                    const C2 ra = rrec[q * GW_RREC + lcy], rb = rrec[(q + 1) * GW_RREC + lcy];
                    R a0, a1, b0, b1;
                    ld2r(crec + q * GW_CREC + lcx, a0, a1);
                    ld2r(crec + (q + 1) * GW_CREC + lcx, b0, b1);
                    acc_cand(lo0, hi0, a0, ra);
                    acc_cand(lo1, hi1, a1, ra);
                    acc_cand(lo0, hi0, b0, rb);
                    acc_cand(lo1, hi1, b1, rb);
                }
                if (q < q1) {
                    const C2 ry = rrec[q * GW_RREC + lcy];
                    R a0, a1;
                    ld2r(crec + q * GW_CREC + lcx, a0, a1);
                    acc_cand(lo0, hi0, a0, ry);
                    acc_cand(lo1, hi1, a1, ry);
                }
                C2* cp = win + (r0 + ((lcy - r0) & 7)) * GW_WP + lcx;
                add2(cp, lo0, lo1);
                add2(cp + 8, hi0, hi1);
            }
            __syncwarp();
        }
        __syncthreads();
        // U += the windows (tile and halo): column ex of the tile window lies in warp
        // ex/8's window (local column ex mod 8) and in warp ex/8 - 1's (local ex mod 8 + 8)
        add_window<R>(Uimg, oy, ox, g, [&](int ey, int ex) {
            const int w0 = ex >> 3, lc = ex & 7;
            C2 sum = mk<C2>(R(0), R(0));
            if (w0 < nw) sum = wins[(size_t)w0 * WS + ey * GW_WP + lc];
            if (w0 >= 1) sum = cadd(sum, wins[(size_t)(w0 - 1) * WS + ey * GW_WP + lc + 8]);
            return sum;
        });
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launchers

template <typename R, int J, int MODE>
static cudaError_t launch_degrid(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out, const DualArgs* a,
                                 const int32_t* tiles, const int32_t* count, int ctas, cudaStream_t s,
                                 int batch = 1) {
    if constexpr (J <= 8)
        if (p->g_mode == PD_G_CSR) return launch_degrid_csr<R, J, MODE>(p, grid, out, a, tiles, count, ctas, s, batch);
    const Geo& g = p->g;
    const int ms = std::max(p->max_tile_segs, 1);
    const size_t win = sizeof(R) == 4 ? (size_t)2 * g.ext * ((g.ext + 2) & ~1) : (size_t)g.ext * g.ext;
    const size_t smem = win * sizeof(cplx_t<R>) + (size_t)16 * ms * sizeof(double) + (size_t)(2 * ms + 1) * sizeof(int);
    cudaError_t e = ensure_smem(k_degrid<R, J, MODE>, smem);
    if (e) return e;
    // CTAs stride over the heaviest-first tile list: launch only as many as are
    // resident at once, so none starts its share late
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid<R, J, MODE>, 256, smem) == cudaSuccess &&
        per_sm > 0)
        ctas = std::min(ctas, per_sm * p->num_sms);
    if ((e = cudaMemsetAsync(p->sched + 4, 0, sizeof(int32_t), s))) return e;
    k_degrid<R, J, MODE><<<ctas, 256, smem, s>>>(
        grid, out, a ? (const cplx_t<R>*)a->y : nullptr, a ? (const cplx_t<R>*)a->v : nullptr,
        (cplx_t<R>*)p->rbuf, p->cell, (const R*)p->fx, (const R*)p->fy, p->perm, p->seg_start, p->seg_block,
        p->tile_seg_start, a ? a->block_active : nullptr, tiles, count, p->seg_part, ms, g, R(2.0 / g.J),
        R(g.beta), p->kbpoly, p->sched + 4, batch, (int64_t)(g.nx / 4 + 1) * 4 * g.Ky, (int64_t)p->M);
    return cudaGetLastError();
}

template <typename R>
cudaError_t degrid_plain(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out_user, cudaStream_t s, int batch) {
    const int ctas = (int)std::min<int64_t>((int64_t)p->g.ntiles * batch, (int64_t)p->num_sms * 8);
    cudaError_t e = cudaSuccess;
    PD_J_DISPATCH(p->g.J, (e = launch_degrid<R, JJ, 0>(p, grid, out_user, nullptr, p->tile_order,
                                                        p->counts_all + 1, ctas, s, batch)));
    return e;
}

template <typename R>
cudaError_t degrid_dual(const pd_plan* p, const cplx_t<R>* grid, const DualArgs& a, const int32_t* tiles,
                        const int32_t* counts, cudaStream_t s) {
    const int ctas = std::min(p->g.ntiles, p->num_sms * 8);
    cudaError_t e = cudaSuccess;
    prof_mark(PH_DEGRID, 0, s);
    PD_J_DISPATCH(p->g.J, (e = launch_degrid<R, JJ, 1>(p, grid, nullptr, &a, tiles, counts + 1, ctas, s)));
    prof_mark(PH_DEGRID, 1, s);
    if (e) return e;
    prof_mark(PH_NORMS, 0, s);
    k_block_norms<R><<<(p->d * 32 + 127) / 128, 128, 0, s>>>(p->seg_part, p->block_seg_start, p->block_seg_list,
                                                       a.block_active, a.eps, p->blk_norm, (R*)p->blk_scale,
                                                       a.res_norm, p->d, 0);
    prof_mark(PH_NORMS, 1, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t degrid_res_norms(const pd_plan* p, const cplx_t<R>* grid, const cplx_t<R>* y, double* res_norm,
                             cudaStream_t s) {
    // every block: the residual part of the pd-mode pass (its r output goes to the
    // plan's scratch and v is not needed, so y stands in for it), then ||G_i b - y_i||
    const int ctas = std::min(p->g.ntiles, p->num_sms * 8);
    DualArgs a{y, (void*)y, nullptr, nullptr, res_norm};
    cudaError_t e = cudaSuccess;
    PD_J_DISPATCH(p->g.J, (e = launch_degrid<R, JJ, 1>(p, grid, nullptr, &a, p->tile_order, p->counts_all + 1,
                                                        ctas, s)));
    if (e) return e;
    k_block_norms<R><<<(p->d * 32 + 127) / 128, 128, 0, s>>>(p->seg_part, p->block_seg_start, p->block_seg_list,
                                                       nullptr, nullptr, nullptr, nullptr, res_norm, p->d, 1);
    return cudaGetLastError();
}

template <typename R, int J, int MODE>
static cudaError_t launch_grid_j(const pd_plan* p, const cplx_t<R>* src, const DualArgs* a, const int32_t* tiles,
                                 const int32_t* count, cplx_t<R>* U, int* next_tile, cudaStream_t s, int batch) {
    if constexpr (J <= 8)
        if (p->g_mode == PD_G_CSR) return launch_grid_csr<R, J, MODE>(p, src, a, tiles, count, U, next_tile, s, batch);
    const Geo& g = p->g;
    const int ms = std::max(p->max_tile_segs, 1);
    const size_t lists = (size_t)(2 * ms + 1) * sizeof(int);
    const R toj = R(2.0 / g.J), beta = R(g.beta);
    const int ctas = std::min(g.ntiles, p->num_sms * 4);
    const cplx_t<R>* rb = (const cplx_t<R>*)p->rbuf;
    cplx_t<R>* vv = a ? (cplx_t<R>*)a->v : nullptr;
    const int32_t* act = a ? a->block_active : nullptr;
    cudaError_t e;
    if constexpr (J <= 8) {
        const int nw = std::max(1, g.tile / SC);
        const size_t smem8 = grid8w_smem<R>(g.tile, nw, ms);
        if ((e = ensure_smem(k_grid8w<R, J, MODE>, smem8))) return e;
        int per_sm = 0;
        int ctas8 = std::min(g.ntiles * batch, p->num_sms * 16);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid8w<R, J, MODE>, nw * 32, smem8) ==
                cudaSuccess && per_sm > 0)
            ctas8 = std::min(ctas8, per_sm * p->num_sms);
        k_grid8w<R, J, MODE><<<ctas8, nw * 32, smem8, s>>>(
            src, rb, vv, (const R*)p->blk_scale, act, p->cell, (const R*)p->fx, (const R*)p->fy, p->perm,
            p->seg_start, p->seg_block, p->tile_seg_start, p->seg_sc_start, tiles, count, U, ms, g, toj, beta,
            p->kbpoly, next_tile, batch, (int64_t)p->M, (int64_t)g.Kx * g.Ky);
    } else {
        const size_t smem = (size_t)2 * g.ext * g.ext * sizeof(R) + lists;
        if ((e = ensure_smem(k_grid<R, J, MODE>, smem))) return e;
        for (int b = 0; b < batch; ++b)        // kernels wider than 8: one launch per image
            k_grid<R, J, MODE><<<ctas, 256, smem, s>>>(src ? src + (int64_t)b * p->M : src, rb, vv,
                                                      (const R*)p->blk_scale, act, p->cell, (const R*)p->fx,
                                                      (const R*)p->fy, p->perm, p->seg_start, p->seg_block,
                                                      p->tile_seg_start, tiles, count,
                                                      U + (int64_t)b * g.Kx * g.Ky, ms, g, toj, beta, p->kbpoly);
    }
    return cudaGetLastError();
}

// One launch per tile colour (their windows are disjoint within a colour), each taking
// its tiles from a dynamically claimed position of its list.
template <typename R>
static cudaError_t launch_grid(const pd_plan* p, int mode, const cplx_t<R>* src, const DualArgs* a,
                               const int32_t* const* tiles, const int32_t* counts4, cplx_t<R>* U, cudaStream_t s,
                               int batch = 1) {
    const Geo& g = p->g;
    cudaError_t e = cudaSuccess;
    prof_mark(PH_GRID, 0, s);
    if ((e = cudaMemsetAsync(p->sched, 0, 4 * sizeof(int32_t), s))) return e;
    for (int c = 0; c < 4 && !e; ++c) {
        if (mode == 0) {
            PD_J_DISPATCH(g.J, (e = launch_grid_j<R, JJ, 0>(p, src, a, tiles[c], counts4 + c, U, p->sched + c, s,
                                                            batch)));
        } else {
            PD_J_DISPATCH(g.J, (e = launch_grid_j<R, JJ, 1>(p, src, a, tiles[c], counts4 + c, U, p->sched + c, s,
                                                            1)));
        }
    }
    prof_mark(PH_GRID, 1, s);
    return e ? e : cudaGetLastError();
}

template <typename R>
cudaError_t grid_plain(const pd_plan* p, const cplx_t<R>* y_user, cplx_t<R>* U, cudaStream_t s, int batch) {
    // U = G^T y: every window is added to a zeroed grid
    cudaError_t e = cudaMemsetAsync(U, 0, (size_t)batch * p->g.Kx * p->g.Ky * sizeof(cplx_t<R>), s);
    if (e) return e;
    const int q = p->g.ntiles / 4;
    const int32_t* lists[4] = {p->colour_tiles, p->colour_tiles + q, p->colour_tiles + 2 * q, p->colour_tiles + 3 * q};
    return launch_grid<R>(p, 0, y_user, nullptr, lists, p->colour_counts, U, s, batch);
}

template <typename R>
cudaError_t grid_dual(const pd_plan* p, const DualArgs& a, const int32_t* const* tiles, const int32_t* counts4,
                      cplx_t<R>* U, cudaStream_t s) {
    return launch_grid<R>(p, 1, nullptr, &a, tiles, counts4, U, s);
}

template cudaError_t degrid_plain<float>(const pd_plan*, const float2*, float2*, cudaStream_t, int);
template cudaError_t degrid_plain<double>(const pd_plan*, const double2*, double2*, cudaStream_t, int);
template cudaError_t degrid_res_norms<float>(const pd_plan*, const float2*, const float2*, double*, cudaStream_t);
template cudaError_t degrid_res_norms<double>(const pd_plan*, const double2*, const double2*, double*, cudaStream_t);
template cudaError_t degrid_dual<float>(const pd_plan*, const float2*, const DualArgs&, const int32_t*,
                                        const int32_t*, cudaStream_t);
template cudaError_t degrid_dual<double>(const pd_plan*, const double2*, const DualArgs&, const int32_t*,
                                         const int32_t*, cudaStream_t);
template cudaError_t grid_plain<float>(const pd_plan*, const float2*, float2*, cudaStream_t, int);
template cudaError_t grid_plain<double>(const pd_plan*, const double2*, double2*, cudaStream_t, int);
template cudaError_t grid_dual<float>(const pd_plan*, const DualArgs&, const int32_t* const*, const int32_t*,
                                      float2*, cudaStream_t);
template cudaError_t grid_dual<double>(const pd_plan*, const DualArgs&, const int32_t* const*, const int32_t*,
                                       double2*, cudaStream_t);

}  // namespace pdgb
