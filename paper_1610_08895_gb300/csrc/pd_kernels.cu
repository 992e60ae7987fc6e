// Small device-resident steps of Algorithm 1: the active-set draws (step 3) with
// the optional adaptive probabilities (Sec. 4, eq. prob-choice), the compaction of
// the active work lists for the persistent degridding/gridding launches, FP64
// reductions, and index permutations between user and internal visibility order.
#include <algorithm>

#include "common.cuh"
#include "plan.hpp"

namespace pdgb {

constexpr int SEL_NT = 1024;

// Exclusive scan of per-thread counts over a 1024-thread block; returns the total.
__device__ int block_excl_scan(int v, int* sh, int& excl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const int before = warp > 0 ? sh[warp - 1] : 0;
    excl = before + x - v;
    const int total = sh[31];
    __syncthreads();
    return total;
}

// Step 3: Philox draws u(seed, t, stream, index) < p for blocks (stream 0) and
// bases (stream 1); with adaptive = 1 the block probabilities are first set by
// eq. (prob-choice) from the current residual norms. Then the tiles holding a
// visibility of an active block are compacted, heaviest first, into the list read
// by the persistent degridding and gridding launches.
__global__ void __launch_bounds__(SEL_NT) k_select(
    uint64_t seed, int adaptive, double an, double pmin, double pmax, int64_t* __restrict__ tptr,
    double* __restrict__ p_block, const double* __restrict__ p_basis, const double* __restrict__ res_norm,
    const double* __restrict__ eps, int d, int b, int32_t* __restrict__ block_active,
    int32_t* __restrict__ basis_active, const int32_t* __restrict__ tile_order,
    const int32_t* __restrict__ tile_seg_start, const int32_t* __restrict__ seg_block, int ntiles,
    int32_t* __restrict__ tile_active, int32_t* __restrict__ act_tiles, int32_t* __restrict__ act_col, int ntx,
    int32_t* __restrict__ counts) {
    __shared__ int shi[32];
    __shared__ double shd[32];
    __shared__ double q_sh, cap_sh;
    __shared__ int64_t t_sh;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int64_t t = *tptr + 1;
        *tptr = t;
        t_sh = t;
    }
    if (adaptive) {
        // c_i = max(||r_i|| - eps_i, 0)^2 / eps_i^2; p_i = p_min + min(q_i + a, p_max - p_min)
        double csum = 0.0;
        for (int i = tid; i < d; i += SEL_NT) {
            const double e = eps[i], r = res_norm[i];
            const double c = r > e ? (r - e) * (r - e) / (e * e) : 0.0;
            csum += c;
        }
        csum = block_sum(csum, shd);
        if (tid == 0) shd[0] = csum;
        __syncthreads();
        csum = shd[0];
        __syncthreads();
        const double cap = pmax - pmin;
        const double target = an - d * pmin;
        if (csum == 0.0) {
            for (int i = tid; i < d; i += SEL_NT) p_block[i] = an / d;
        } else {
            const double qs = target / csum;
            // a = 0 unless some q_i exceeds the cap (then some p_i saturates at p_max)
            int sat = 0;
            for (int i = tid; i < d; i += SEL_NT) {
                const double e = eps[i], r = res_norm[i];
                const double c = r > e ? (r - e) * (r - e) / (e * e) : 0.0;
                sat |= (qs * c > cap);
            }
            sat = __syncthreads_or(sat);
            double lo = 0.0, hi = 0.0;
            if (sat) {
                // f(a) = sum min(q_i + a, cap) is non-decreasing: bisection to double precision
                hi = cap;
                for (int it = 0; it < 80; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    double f = 0.0;
                    for (int i = tid; i < d; i += SEL_NT) {
                        const double e = eps[i], r = res_norm[i];
                        const double c = r > e ? (r - e) * (r - e) / (e * e) : 0.0;
                        f += fmin(qs * c + mid, cap);
                    }
                    f = block_sum(f, shd);
                    if (tid == 0) shd[0] = f;
                    __syncthreads();
                    f = shd[0];
                    __syncthreads();
                    if (f < target) lo = mid; else hi = mid;
                }
            }
            if (tid == 0) { q_sh = qs; cap_sh = hi; }
            __syncthreads();
            const double a = cap_sh;
            for (int i = tid; i < d; i += SEL_NT) {
                const double e = eps[i], r = res_norm[i];
                const double c = r > e ? (r - e) * (r - e) / (e * e) : 0.0;
                p_block[i] = pmin + fmin(q_sh * c + a, cap);
            }
        }
    }
    __syncthreads();
    const int64_t t = t_sh;
    for (int i = tid; i < d; i += SEL_NT) block_active[i] = philox_uniform(seed, (uint64_t)t, 0, i) < p_block[i];
    for (int j = tid; j < b; j += SEL_NT) basis_active[j] = philox_uniform(seed, (uint64_t)t, 1, j) < p_basis[j];
    __syncthreads();
    // active tiles, in the static heaviest-first order (all of them for the degridding,
    // and split by colour for the gridding); count active segments too
    {
        const int per = (ntiles + SEL_NT - 1) / SEL_NT;
        const int k0 = min(ntiles, tid * per), k1 = min(ntiles, k0 + per);
        int mine = 0, segs = 0, mc[4] = {0, 0, 0, 0};
        // the flags of this thread's tiles, kept in registers for the compaction pass
        // below (up to 128 tiles per thread; beyond that it reads tile_active back)
        constexpr int FW = 4;
        uint32_t onm[FW] = {0u, 0u, 0u, 0u};
        // batches of tiles whose independent loads go out together
        constexpr int TB = 8;
        for (int kb = k0; kb < k1; kb += TB) {
            int tt[TB], s0[TB], s1[TB];
#pragma unroll
            for (int i = 0; i < TB; ++i) tt[i] = kb + i < k1 ? tile_order[kb + i] : -1;
#pragma unroll
            for (int i = 0; i < TB; ++i) {
                s0[i] = tt[i] >= 0 ? tile_seg_start[tt[i]] : 0;
                s1[i] = tt[i] >= 0 ? tile_seg_start[tt[i] + 1] : 0;
            }
#pragma unroll
            for (int i = 0; i < TB; ++i) {
                if (tt[i] < 0) continue;
                int on = 0;
                for (int sg = s0[i]; sg < s1[i]; ++sg) {
                    const int a = block_active[seg_block[sg]];
                    on |= a;
                    segs += a;
                }
                tile_active[tt[i]] = on;
                const int li = kb + i - k0;
#pragma unroll
                for (int f = 0; f < FW; ++f)
                    if (on && (li >> 5) == f) onm[f] |= 1u << (li & 31);
                mine += on;
                const int col = tile_colour(tt[i], ntx);
#pragma unroll
                for (int c = 0; c < 4; ++c) mc[c] += on && col == c;
            }
        }
        int excl, sexcl, cex[4];
        const int total = block_excl_scan(mine, shi, excl);
        const int stotal = block_excl_scan(segs, shi, sexcl);
        int ctot[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ctot[c] = block_excl_scan(mc[c], shi, cex[c]);
        const int q = ntiles / 4;
        for (int k = k0; k < k1; ++k) {
            const int li = k - k0;
            bool on;
            if (li < 32 * FW) {
                uint32_t w = onm[0];
#pragma unroll
                for (int f = 1; f < FW; ++f) w = (li >> 5) == f ? onm[f] : w;
                on = (w >> (li & 31)) & 1u;
            } else {
                on = tile_active[tile_order[k]];
            }
            if (on) {
                const int tt = tile_order[k];
                act_tiles[excl++] = tt;
                const int col = tile_colour(tt, ntx);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (col == c) act_col[c * q + cex[c]++] = tt;
            }
        }
        if (tid == 0) {
            counts[0] = stotal;
            counts[1] = total;
#pragma unroll
            for (int c = 0; c < 4; ++c) counts[2 + c] = ctot[c];
        }
    }
}

cudaError_t select_active(const pd_plan* p, pd_state* st, const SelectArgs& a, cudaStream_t s) {
    prof_mark(PH_SELECT, 0, s);
    k_select<<<1, SEL_NT, 0, s>>>(a.seed, a.adaptive, a.n, a.p_min, a.p_max, st->t, st->p_block, st->p_basis,
                                 st->res_norm, st->eps, p->d, p->b, st->block_active, st->basis_active,
                                 p->tile_order, p->tile_seg_start, p->seg_block, p->g.ntiles,
                                 st->tile_active, st->act_tiles, st->act_col, p->g.ntx, st->counts);
    prof_mark(PH_SELECT, 1, s);
    return cudaGetLastError();
}

// Fixed-order sum of per-CTA partials of the primal update: ||x^t - x^{t-1}||^2, ||x^t||^2.
__global__ void k_sum_pairs(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

cudaError_t primal_finish(const pd_plan* p, pd_state* st, cudaStream_t s) {
    prof_mark(PH_FINISH, 0, s);
    k_sum_pairs<<<1, 256, 0, s>>>(st->prim_part, inv_rows_ctas(p), st->diag);
    prof_mark(PH_FINISH, 1, s);
    return cudaGetLastError();
}

// Deterministic two-level FP64 sum of squares.
template <typename R>
__global__ void k_sq_part(const R* __restrict__ x, int64_t n, double* __restrict__ part) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a += (double)x[i] * (double)x[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}
__global__ void k_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) *out = a;
}

template <typename R>
cudaError_t norm2(const pd_plan* p, const R* x, int64_t n, double* out, cudaStream_t s) {
    const int ctas = std::min<int64_t>(p->red_len, std::max<int64_t>(1, (n + 255) / 256));
    k_sq_part<R><<<ctas, 256, 0, s>>>(x, n, p->red);
    k_sum<<<1, 256, 0, s>>>(p->red, ctas, out);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_scale_copy(const R* __restrict__ x, R* __restrict__ y, int64_t n, R scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * scale;
}
template <typename R>
cudaError_t scale_copy(const R* x, R* y, int64_t n, double scale, cudaStream_t s) {
    const int ctas = (int)std::min<int64_t>(4096, (n + 255) / 256);
    k_scale_copy<R><<<ctas, 256, 0, s>>>(x, y, n, (R)scale);
    return cudaGetLastError();
}

template <typename C>
__global__ void k_gather(const C* __restrict__ user, C* __restrict__ internal, const int32_t* __restrict__ perm,
                         int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        internal[i] = user[perm[i]];
}
template <typename C>
__global__ void k_scatter(const C* __restrict__ internal, C* __restrict__ user, const int32_t* __restrict__ perm,
                          int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        user[perm[i]] = internal[i];
}
template <typename R>
cudaError_t gather_internal(const pd_plan* p, const cplx_t<R>* user, cplx_t<R>* internal, cudaStream_t s) {
    const int ctas = (int)std::min<int64_t>(4096, (p->M + 255) / 256);
    k_gather<<<ctas, 256, 0, s>>>(user, internal, p->perm, p->M);
    return cudaGetLastError();
}
template <typename R>
cudaError_t scatter_user(const pd_plan* p, const cplx_t<R>* internal, cplx_t<R>* user, cudaStream_t s) {
    const int ctas = (int)std::min<int64_t>(4096, (p->M + 255) / 256);
    k_scatter<<<ctas, 256, 0, s>>>(internal, user, p->perm, p->M);
    return cudaGetLastError();
}

// ||y_i|| per block (= ||Phi_i x^(0) - y_i|| for x^(0) = 0): segment partials, then
// a fixed-order sum per block.
template <typename R>
__global__ void k_seg_sq(const cplx_t<R>* __restrict__ y, const int32_t* __restrict__ seg_start, int nseg,
                         double* __restrict__ part) {
    __shared__ double sh[32];
    for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        double a = 0.0;
        for (int m = seg_start[sg] + threadIdx.x; m < seg_start[sg + 1]; m += blockDim.x)
            a += (double)y[m].x * y[m].x + (double)y[m].y * y[m].y;
        a = block_sum(a, sh);
        if (threadIdx.x == 0) part[2 * sg + 1] = a;
    }
}
__global__ void k_block_sqrt(const double* __restrict__ part, const int32_t* __restrict__ bss,
                             const int32_t* __restrict__ bsl, int d, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double a = 0.0;
    for (int k = bss[i]; k < bss[i + 1]; ++k) a += part[2 * bsl[k] + 1];
    out[i] = sqrt(a);
}
cudaError_t init_res_norm(const pd_plan* p, pd_state* st, cudaStream_t s) {
    const int ctas = (int)std::min<int64_t>(std::max<int64_t>(p->nseg, 1), (int64_t)p->num_sms * 8);
    if (p->prec == PD_F64)
        k_seg_sq<double><<<ctas, 256, 0, s>>>((const double2*)st->y, p->seg_start, (int)p->nseg, p->seg_part);
    else
        k_seg_sq<float><<<ctas, 256, 0, s>>>((const float2*)st->y, p->seg_start, (int)p->nseg, p->seg_part);
    k_block_sqrt<<<(p->d + 127) / 128, 128, 0, s>>>(p->seg_part, p->block_seg_start, p->block_seg_list, p->d,
                                                    st->res_norm);
    return cudaGetLastError();
}

// Synthesis form, dual of positivity and the image-domain term of the primal step:
// u <- min(u + x~, 0) (z - P_C(z)); back <- sigma u + varsigma back.
template <typename R>
__global__ void k_synth_dual(const R* __restrict__ xt, R* __restrict__ u, R* __restrict__ back, int64_t n, R sigma,
                             R varsigma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R z = u[i] + xt[i];
        const R un = z < R(0) ? z : R(0);
        u[i] = un;
        back[i] = sigma * un + varsigma * back[i];
    }
}

// Synthesis form, primal step on the coefficients: alpha_new = S_thr(alpha - tau w)
// (eq. prox-L1), alpha~ = 2 alpha_new - alpha, alpha = alpha_new.
template <typename R>
__global__ void k_synth_primal(R* __restrict__ alpha, R* __restrict__ alpha_t, const R* __restrict__ w, int64_t n,
                               R tau, R thr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R a = alpha[i];
        const R q = a - tau * w[i];
        const R an = q > thr ? q - thr : (q < -thr ? q + thr : R(0));
        alpha_t[i] = R(2) * an - a;
        alpha[i] = an;
    }
}

template <typename R>
cudaError_t synth_dual(const pd_plan* p, const R* xt, R* u, R* back, double sigma, double varsigma, cudaStream_t s) {
    const int64_t n = (int64_t)p->g.nx * p->g.ny;
    const int ctas = (int)std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8);
    k_synth_dual<R><<<ctas, 256, 0, s>>>(xt, u, back, n, (R)sigma, (R)varsigma);
    return cudaGetLastError();
}

template <typename R>
cudaError_t synth_primal(const pd_plan* p, R* alpha, R* alpha_t, const R* w, double tau, double thr, cudaStream_t s) {
    const int64_t n = (int64_t)p->b * p->g.nx * p->g.ny;
    const int ctas = (int)std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8);
    k_synth_primal<R><<<ctas, 256, 0, s>>>(alpha, alpha_t, w, n, (R)tau, (R)thr);
    return cudaGetLastError();
}

template cudaError_t synth_dual<float>(const pd_plan*, const float*, float*, float*, double, double, cudaStream_t);
template cudaError_t synth_dual<double>(const pd_plan*, const double*, double*, double*, double, double, cudaStream_t);
template cudaError_t synth_primal<float>(const pd_plan*, float*, float*, const float*, double, double, cudaStream_t);
template cudaError_t synth_primal<double>(const pd_plan*, double*, double*, const double*, double, double,
                                          cudaStream_t);
template cudaError_t norm2<float>(const pd_plan*, const float*, int64_t, double*, cudaStream_t);
template cudaError_t norm2<double>(const pd_plan*, const double*, int64_t, double*, cudaStream_t);
template cudaError_t scale_copy<float>(const float*, float*, int64_t, double, cudaStream_t);
template cudaError_t scale_copy<double>(const double*, double*, int64_t, double, cudaStream_t);
template cudaError_t gather_internal<float>(const pd_plan*, const float2*, float2*, cudaStream_t);
template cudaError_t gather_internal<double>(const pd_plan*, const double2*, double2*, cudaStream_t);
template cudaError_t scatter_user<float>(const pd_plan*, const float2*, float2*, cudaStream_t);
template cudaError_t scatter_user<double>(const pd_plan*, const double2*, double2*, cudaStream_t);

}  // namespace pdgb
