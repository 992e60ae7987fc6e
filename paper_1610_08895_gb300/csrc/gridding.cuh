// Device helpers shared by the two forms of the interpolation G: weights evaluated in
// the kernels (gridding.cu) and G stored as a sparse matrix (gridding_csr.cu).
#pragma once
#include "common.cuh"
#include "plan.hpp"

namespace pdgb {

// The J tap weights phi(frac + J/2 - 1 - a) of one axis. FP32: the plan's per-tap
// Chebyshev interpolants (degree 10, interpolation error ~3e-11 of phi(0), below FP32
// resolution) in x = 2 frac - 1. phi is even, so tap J-1-a is tap a at -x: with the
// polynomial split into even and odd parts p = E(x^2) + x O(x^2), one pass gives both
// E + x O (tap a) and E - x O (tap J-1-a). FP64: I0 itself.
template <typename R, int J>
__device__ __forceinline__ void kb_taps(R frac, R* w, R two_over_j, R beta, const KbPoly& kp) {
    if constexpr (sizeof(R) == 4) {
        const float x = 2.0f * frac - 1.0f, x2 = x * x;
#pragma unroll
        for (int a = 0; a < J / 2; ++a) {
            float ev = kp.c[a][KB_DEG], od = kp.c[a][KB_DEG - 1];
#pragma unroll
            for (int k = KB_DEG - 2; k >= 0; k -= 2) ev = fmaf(ev, x2, kp.c[a][k]);
#pragma unroll
            for (int k = KB_DEG - 3; k >= 1; k -= 2) od = fmaf(od, x2, kp.c[a][k]);
            w[a] = fmaf(x, od, ev);
            w[J - 1 - a] = fmaf(-x, od, ev);
        }
    } else {
#pragma unroll
        for (int a = 0; a < J; ++a) w[a] = kb_weight<R>(frac + R(J / 2 - 1 - a), two_over_j, beta);
    }
}

// ---------------------------------------------------------------- active segments
// Warp 0 lists the tile's segments whose block is active (all of them when active is
// null) in act_seg[0..nact) and the prefix sums of their lengths in act_pre[0..nact];
// returns nact to every thread (the caller syncs before use).
__device__ __forceinline__ void list_active_segments(int seg0, int nseg_t, const int32_t* __restrict__ seg_block,
                                                     const int32_t* __restrict__ active,
                                                     const int32_t* __restrict__ seg_start, int* act_seg,
                                                     int* act_pre, int* nact_out) {
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int nact = 0, total = 0;
    for (int base = 0; base < nseg_t; base += 32) {
        const int k = base + lane;
        const bool ok = k < nseg_t && (active == nullptr || active[seg_block[seg0 + k]]);
        const int len = ok ? seg_start[seg0 + k + 1] - seg_start[seg0 + k] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (ok) {
            const int pos = nact + __popc(bal & below);
            act_seg[pos] = seg0 + k;
            act_pre[pos] = total + incl - len;
        }
        total += __shfl_sync(0xffffffffu, incl, 31);
        nact += __popc(bal);
    }
    if (lane == 0) { act_pre[nact] = total; *nact_out = nact; }
}

// Cell (ky, kx) of F Z x from the half grid (columns 0 .. nx, column panels): the image
// is real, so the columns kx > nx are conj(b[-ky][-kx]).
template <typename C2>
__device__ __forceinline__ C2 half_grid_at(const C2* __restrict__ gh, int ky, int kx, const Geo& g) {
    if (kx <= g.nx) return gh[panel_off(ky, kx, g.Ky)];
    const C2 v = gh[panel_off((g.Ky - ky) & (g.Ky - 1), g.Kx - kx, g.Ky)];
    return mk<C2>(v.x, -v.y);
}

// ---------------------------------------------------------------- reductions
// Warp-level segmented sum: the lanes with ok add (a, b) to their local segment ls;
// lane 0 adds each segment's warp total into part[2 ls], part[2 ls + 1] (FP64 slots
// owned by this warp), always in the same order. The at most 32 terms of one warp are
// summed in the working precision A (a fixed shuffle tree of non-negative terms:
// relative error below 6 units of A's rounding), every sum above that in FP64.
template <typename A>
__device__ __forceinline__ void warp_seg_add(bool ok, int ls, A a, A b, double* part) {
    unsigned todo = __ballot_sync(0xffffffffu, ok);
    while (todo) {
        const int key = __shfl_sync(0xffffffffu, ls, __ffs(todo) - 1);
        const bool mine = ok && ls == key;
        const unsigned mask = __ballot_sync(0xffffffffu, mine);
        const A x = warp_sum(mine ? a : A(0)), y = warp_sum(mine ? b : A(0));
        if ((threadIdx.x & 31) == 0) { part[2 * key] += (double)x; part[2 * key + 1] += (double)y; }
        todo &= ~mask;
    }
}

// value of visibility m to grid: MODE 0 the input (user order); MODE 1 the dual change
// v_new - v_old with v_new = scale_i r (step 8), writing v_new.
template <typename R, int MODE>
__device__ __forceinline__ cplx_t<R> grid_value(int m, const cplx_t<R>* __restrict__ src,
                                                const cplx_t<R>* __restrict__ rbuf, cplx_t<R>* __restrict__ v,
                                                const int32_t* __restrict__ perm, R sc) {
    if (MODE == 0) return src[perm[m]];
    const cplx_t<R> r = rbuf[m], vo = v[m];
    const cplx_t<R> vn = cscale(r, sc);
    v[m] = vn;
    return csub(vn, vo);
}

// U += the tile's E x E window (tile and halo, wrapped periodically), the window's value
// of cell (ey, ex) given by val(ey, ex). The U reads of a batch of cells go out together.
template <typename R, class V>
__device__ __forceinline__ void add_window(cplx_t<R>* __restrict__ U, int oy, int ox, const Geo& g, const V& val) {
    using C2 = cplx_t<R>;
    const int E = g.ext, H = g.halo_lo;
    constexpr int EB = 8;
    for (int i0 = threadIdx.x; i0 < E * E; i0 += EB * (int)blockDim.x) {
        C2 uo[EB];
        int64_t off[EB];
#pragma unroll
        for (int k = 0; k < EB; ++k) {
            const int i = i0 + k * (int)blockDim.x;
            off[k] = -1;
            if (i < E * E) {
                const int ey = i / E, ex = i - ey * E;
                off[k] = panel_off((oy - H + ey) & (g.Ky - 1), (ox - H + ex) & (g.Kx - 1), g.Ky);
                uo[k] = U[off[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < EB; ++k) {
            if (off[k] < 0) break;
            const int i = i0 + k * (int)blockDim.x;
            const int ey = i / E, ex = i - ey * E;
            U[off[k]] = cadd(uo[k], val(ey, ex));
        }
    }
}

#define PD_J_DISPATCH(J_, CALL)                          \
    switch (J_) {                                        \
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

// G held as a sparse matrix (gridding_csr.cu), J <= 8: the same contracts as the
// on-the-fly launchers of gridding.cu, which hand over to these when the plan's
// g_mode is PD_G_CSR.
template <typename R, int J, int MODE>
cudaError_t launch_degrid_csr(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out, const DualArgs* a,
                              const int32_t* tiles, const int32_t* count, int ctas, cudaStream_t s, int batch);
template <typename R, int J, int MODE>
cudaError_t launch_grid_csr(const pd_plan* p, const cplx_t<R>* src, const DualArgs* a, const int32_t* tiles,
                            const int32_t* count, cplx_t<R>* U, int* next_tile, cudaStream_t s, int batch);

}  // namespace pdgb
