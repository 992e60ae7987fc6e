// C ABI of the PD-R library (declared in include/pd.h): plan construction (host
// sorting and tables), the operator entry points, the Algorithm 1 state and the
// iteration driver with optional CUDA-graph replay.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "host_math.hpp"
#include "plan.hpp"

using namespace pdgb;

static thread_local std::string g_err = "no error";

static pd_status fail(pd_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CU(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* pd_last_error(void) { return g_err.c_str(); }

pd_status pdgb::set_error(pd_status st, const char* msg) { return fail(st, msg); }

// ---- per-phase CUDA-event timing (pd_params.profile)
static thread_local pd_state* g_prof = nullptr;

void pdgb::prof_mark(int phase, int end, cudaStream_t s) {
    if (!g_prof || phase < 0 || phase >= PH_COUNT) return;
    cudaEventRecord(g_prof->prof_ev[2 * phase + end], s);
}

static const char* k_phase_names[PH_COUNT] = {
    "select", "fwd_rows", "fwd_cols", "degrid_dual", "block_norms", "grid_dual",
    "wavelet_analysis", "wavelet_synthesis", "inv_cols", "inv_rows_primal", "primal_finish"};

extern "C" const char* pd_phase_name(int32_t phase) {
    return phase >= 0 && phase < PH_COUNT ? k_phase_names[phase] : "unknown";
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }

template <typename T> static cudaError_t dalloc(std::vector<void*>& list, size_t& bytes, T** ptr, size_t count) {
    size_t nb = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc((void**)ptr, nb);
    if (e == cudaSuccess) { list.push_back((void*)*ptr); bytes += nb; }
    return e;
}
static cudaError_t dalloc_bytes(std::vector<void*>& list, size_t& bytes, void** ptr, size_t nb) {
    nb = std::max<size_t>(nb, 16);
    cudaError_t e = cudaMalloc(ptr, nb);
    if (e == cudaSuccess) { list.push_back(*ptr); bytes += nb; }
    return e;
}
template <typename T> static cudaError_t upload(T* dst, const std::vector<T>& src) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}
static std::vector<unsigned char> as_real_bytes(const std::vector<double>& v, int prec) {
    std::vector<unsigned char> out;
    if (prec == PD_F64) {
        out.resize(v.size() * sizeof(double));
        std::memcpy(out.data(), v.data(), out.size());
    } else {
        std::vector<float> f(v.begin(), v.end());
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    }
    return out;
}
static cudaError_t upload_real(void* dst, const std::vector<double>& v, int prec) {
    std::vector<unsigned char> b = as_real_bytes(v, prec);
    if (b.empty()) return cudaSuccess;
    return cudaMemcpy(dst, b.data(), b.size(), cudaMemcpyHostToDevice);
}

static void free_all(std::vector<void*>& list) {
    for (void* q : list) cudaFree(q);
    list.clear();
}

extern "C" pd_status pd_plan_destroy(pd_plan* p) {
    if (!p) return PD_OK;
    free_all(p->allocs);
    delete p;
    return PD_OK;
}

extern "C" pd_status pd_daubechies_filter(int32_t k, double* h) {
    if (k < 1 || k > 8 || !h) return fail(PD_EINVAL, "pd_daubechies_filter: k must be in 1..8 and h non-null");
    std::vector<double> f = daubechies(k);
    std::memcpy(h, f.data(), f.size() * sizeof(double));
    return PD_OK;
}

static pd_status plan_build(pd_plan* p, const pd_plan_desc* d);

extern "C" pd_status pd_plan_create(const pd_plan_desc* d, pd_plan** out) {
    if (!d || !out) return fail(PD_EINVAL, "pd_plan_create: null argument");
    *out = nullptr;
    pd_plan* p = new pd_plan();
    pd_status st = plan_build(p, d);
    if (st != PD_OK) {
        pd_plan_destroy(p);
        return st;
    }
    *out = p;
    return PD_OK;
}

static pd_status plan_build(pd_plan* p, const pd_plan_desc* d) {
    if (!is_pow2(d->nx) || !is_pow2(d->ny) || d->nx < 16 || d->ny < 16 || d->nx > 8192 || d->ny > 8192)
        return fail(PD_EINVAL, "image sides must be powers of two in [16, 8192]");
    if (d->osf != 2) return fail(PD_EINVAL, "oversampling per axis must be 2");
    if (d->precision == PD_F64 && (d->nx > 4096 || d->ny > 4096))
        return fail(PD_ENOTSUP, "FP64 plans support image sides up to 4096");
    if (d->nvis < 1 || d->nvis > (int64_t)0x7fffffff) return fail(PD_EINVAL, "nvis must be in [1, 2^31)");
    if (!d->uv || !d->block_of_vis) return fail(PD_EINVAL, "uv and block_of_vis must be non-null");
    if (d->nblocks < 1 || d->nblocks > 4096) return fail(PD_EINVAL, "nblocks must be in [1, 4096]");
    if (d->kernel_width < 2 || d->kernel_width > 16 || (d->kernel_width & 1))
        return fail(PD_EINVAL, "kernel_width must be even in [2, 16]");
    if (d->nbases < 1 || d->nbases > MAX_BASES || !d->basis_ids) return fail(PD_EINVAL, "nbases must be in [1, 16]");
    for (int k = 0; k < d->nbases; ++k)
        if (d->basis_ids[k] < 0 || d->basis_ids[k] > 8) return fail(PD_EINVAL, "basis ids must be 0 (Dirac) or 1..8");
    // bounded before the shift test (a shift by 32 or more is undefined)
    if (d->levels < 1 || d->levels > 13 || (d->nx >> d->levels) < 1 || (d->ny >> d->levels) < 1)
        return fail(PD_EINVAL, "levels must satisfy 1 <= L <= 13 and n >> L >= 1");
    if (d->precision != PD_F32 && d->precision != PD_F64) return fail(PD_EINVAL, "precision must be PD_F32 or PD_F64");
    if (d->kb_beta < 0) return fail(PD_EINVAL, "kb_beta must be >= 0");
    const int dde = d->dde_width > 1 ? d->dde_width : 0;
    if (d->dde_width < 0 || (dde && ((dde & 1) == 0 || !d->dde_kernels)))
        return fail(PD_EINVAL, "dde_width must be 0, 1 or odd >= 3 with dde_kernels given");
    if (dde && d->g_mode != PD_G_CSR) return fail(PD_EINVAL, "DDE-aware G needs g_mode = PD_G_CSR");
    if (dde && d->kernel_width + dde - 1 > 8)
        return fail(PD_ENOTSUP, "DDE-aware G needs kernel_width + dde_width - 1 <= 8");
    const int Jfoot = d->kernel_width + (dde ? dde - 1 : 0);   // footprint width of a row of G
    if (d->tile != 0 && (!is_pow2(d->tile) || d->tile < Jfoot))
        return fail(PD_EINVAL, "tile must be 0 or a power of two >= the kernel footprint");
    if (d->g_mode != PD_G_ON_THE_FLY && d->g_mode != PD_G_CSR)
        return fail(PD_EINVAL, "g_mode must be PD_G_ON_THE_FLY or PD_G_CSR");
    if (d->g_mode == PD_G_CSR && d->kernel_width > 8) return fail(PD_ENOTSUP, "the CSR form of G needs J <= 8");

    p->prec = d->precision;
    p->g_mode = d->g_mode;
    p->rsz = p->prec == PD_F64 ? 8 : 4;
    p->csz = 2 * p->rsz;
    Geo& g = p->g;
    g.nx = d->nx; g.ny = d->ny; g.Kx = 2 * d->nx; g.Ky = 2 * d->ny;
    p->kb_J = d->kernel_width;
    p->dde = dde;
    p->csr_cplx = dde > 0;
    g.J = Jfoot;   // tiles, windows and halos follow the footprint; weights use kb_J
    g.beta = d->kb_beta > 0 ? d->kb_beta : kb_beta_default(p->kb_J);
    // default tile: 32 cells (the densest tiles bound the gridding critical path); at least
    // two tiles per grid side, for the colour classes of the gridding
    int T = d->tile ? d->tile : 32;
    while (T > std::min(g.Kx, g.Ky) / 2) T >>= 1;
    while (T < g.J) T <<= 1;
    if (T > std::min(g.Kx, g.Ky) / 2) return fail(PD_ENOTSUP, "grid side below twice the kernel width");
    g.tile = T; g.logT = ilog2(T);
    g.ntx = g.Kx / T; g.nty = g.Ky / T; g.ntiles = g.ntx * g.nty;
    g.ext = T + g.J - 1; g.halo_lo = g.J / 2 - 1; g.halo_hi = g.J / 2;
    p->M = d->nvis; p->d = d->nblocks; p->b = d->nbases; p->L = d->levels;
    p->basis_ids.assign(d->basis_ids, d->basis_ids + d->nbases);
    p->n_wavelet = 0;
    for (int id : p->basis_ids) p->n_wavelet += id > 0;
    CU(cudaGetDevice(&p->device));
    CU(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));

    // ---- visibilities: base cell, fraction, (tile, block) order
    const int64_t M = p->M;
    std::vector<int32_t> bx(M), by(M);
    std::vector<double> frx(M), fry(M);
    for (int64_t m = 0; m < M; ++m) {
        const double u = d->uv[2 * m], v = d->uv[2 * m + 1];
        if (!(u >= -M_PI && u < M_PI && v >= -M_PI && v < M_PI))
            return fail(PD_EINVAL, "uv points must lie in [-pi, pi)^2");
        const int blk = d->block_of_vis[m];
        if (blk < 0 || blk >= p->d) return fail(PD_EINVAL, "block_of_vis out of range");
        const double gxv = u * g.Kx / (2.0 * M_PI), gyv = v * g.Ky / (2.0 * M_PI);
        double flx = std::floor(gxv), fly = std::floor(gyv);
        double fx = gxv - flx, fy = gyv - fly;
        // a fraction that rounds to 1 in the working precision moves to the next cell
        if (p->prec == PD_F32) {
            if ((float)fx >= 1.0f) { flx += 1.0; fx = 0.0; }
            if ((float)fy >= 1.0f) { fly += 1.0; fy = 0.0; }
        }
        bx[m] = (int32_t)((((int64_t)flx % g.Kx) + g.Kx) % g.Kx);
        by[m] = (int32_t)((((int64_t)fly % g.Ky) + g.Ky) % g.Ky);
        frx[m] = fx;
        fry[m] = fy;
    }
    const int64_t nbucket = (int64_t)g.ntiles * p->d;
    std::vector<int32_t> order(M);
    {
        std::vector<int64_t> key(M);
        for (int64_t m = 0; m < M; ++m) {
            const int t = (by[m] >> g.logT) * g.ntx + (bx[m] >> g.logT);
            key[m] = (int64_t)t * p->d + d->block_of_vis[m];
        }
        if (nbucket <= (int64_t)1 << 25) {
            std::vector<int64_t> cnt(nbucket + 1, 0);
            for (int64_t m = 0; m < M; ++m) cnt[key[m] + 1]++;
            for (int64_t k = 0; k < nbucket; ++k) cnt[k + 1] += cnt[k];
            for (int64_t m = 0; m < M; ++m) order[cnt[key[m]]++] = (int32_t)m;
        } else {
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b2) { return key[a] < key[b2]; });
        }
        // segments = runs of equal (tile, block)
        std::vector<int32_t> seg_start, seg_block, seg_tile;
        int64_t prev = -1;
        for (int64_t i = 0; i < M; ++i) {
            const int64_t k = key[order[i]];
            if (k != prev) {
                seg_start.push_back((int32_t)i);
                seg_block.push_back((int32_t)(k % p->d));
                seg_tile.push_back((int32_t)(k / p->d));
                prev = k;
            }
        }
        p->nseg = (int64_t)seg_block.size();
        seg_start.push_back((int32_t)M);
        std::vector<int32_t> tile_seg_start(g.ntiles + 1, 0);
        {
            int64_t s = 0;
            for (int t = 0; t <= g.ntiles; ++t) {
                while (s < p->nseg && seg_tile[s] < t) ++s;
                tile_seg_start[t] = (int32_t)s;
            }
        }
        p->max_tile_segs = 0;
        for (int t = 0; t < g.ntiles; ++t)
            p->max_tile_segs = std::max(p->max_tile_segs, tile_seg_start[t + 1] - tile_seg_start[t]);
        if (p->max_tile_segs > 1024)
            return fail(PD_ENOTSUP, "more than 1024 blocks share one gridding tile; use a smaller tile");
        // within each segment: by 8 x 8 super-cell, then row-major by base cell (stable: ties
        // keep user order), so that the points of one super-cell row are consecutive
        p->nsc_side = std::max(1, g.tile / SC);
        auto scell_of = [&](int32_t m) {
            const int ly = by[m] & (g.tile - 1), lx = bx[m] & (g.tile - 1);
            return (ly / SC) * p->nsc_side + lx / SC;
        };
        const int nsc = p->nsc_side * p->nsc_side;
        std::vector<int32_t> sc_start((size_t)p->nseg * (nsc + 1));
        for (int64_t sg = 0; sg < p->nseg; ++sg) {
            std::stable_sort(order.begin() + seg_start[sg], order.begin() + seg_start[sg + 1],
                             [&](int32_t a, int32_t b2) {
                                 const int sa = scell_of(a), sb = scell_of(b2);
                                 if (sa != sb) return sa < sb;
                                 return (by[a] != by[b2]) ? by[a] < by[b2] : bx[a] < bx[b2];
                             });
            // start of each super-cell's points inside the segment (the gridding's per-warp ranges)
            int32_t* o = &sc_start[(size_t)sg * (nsc + 1)];
            int i = seg_start[sg];
            for (int k = 0; k <= nsc; ++k) {
                while (i < seg_start[sg + 1] && scell_of(order[i]) < k) ++i;
                o[k] = i;
            }
        }
        p->h_sc_start = std::move(sc_start);
        // segments of each block (tile order) for the fixed-order block reductions
        std::vector<int32_t> bss(p->d + 1, 0), bsl(p->nseg);
        for (int64_t sg = 0; sg < p->nseg; ++sg) bss[seg_block[sg] + 1]++;
        for (int i = 0; i < p->d; ++i) bss[i + 1] += bss[i];
        {
            std::vector<int32_t> fill(bss.begin(), bss.end() - 1);
            for (int64_t sg = 0; sg < p->nseg; ++sg) bsl[fill[seg_block[sg]]++] = (int32_t)sg;
        }
        // tiles by decreasing visibility count (heaviest scheduled first)
        std::vector<int32_t> tord(g.ntiles);
        std::iota(tord.begin(), tord.end(), 0);
        auto tcount = [&](int32_t t) { return seg_start[tile_seg_start[t + 1]] - seg_start[tile_seg_start[t]]; };
        std::stable_sort(tord.begin(), tord.end(), [&](int32_t a, int32_t b2) { return tcount(a) > tcount(b2); });
        p->ntiles_nonempty = 0;
        for (int t = 0; t < g.ntiles; ++t) p->ntiles_nonempty += tcount(t) > 0;
        p->h_tile_seg_start = tile_seg_start;
        p->h_seg_block = seg_block;
        p->h_block_seg_start = bss;
        p->h_block_seg_list = bsl;

        auto& A = p->allocs;
        size_t& B = p->device_bytes;
#define ALLOC(ptr, count) CU(dalloc(A, B, &(ptr), (count)))
        ALLOC(p->seg_start, seg_start.size());
        ALLOC(p->seg_block, seg_block.size());
        ALLOC(p->tile_seg_start, tile_seg_start.size());
        ALLOC(p->block_seg_start, bss.size());
        ALLOC(p->block_seg_list, bsl.size());
        ALLOC(p->tile_order, tord.size());
        ALLOC(p->seg_sc_start, p->h_sc_start.size());
        CU(upload(p->seg_sc_start, p->h_sc_start));
        p->h_sc_start.clear();
        p->h_sc_start.shrink_to_fit();
        {
            // tiles of each colour in heaviest-first order
            const int q = g.ntiles / 4;
            std::vector<int32_t> col((size_t)g.ntiles), fill(4, 0), cc(4, q);
            for (int k = 0; k < g.ntiles; ++k) {
                const int c = tile_colour(tord[k], g.ntx);
                col[(size_t)c * q + fill[c]++] = tord[k];
            }
            ALLOC(p->colour_tiles, col.size());
            ALLOC(p->colour_counts, 4);
            CU(upload(p->colour_tiles, col));
            CU(upload(p->colour_counts, cc));
        }
        CU(upload(p->seg_start, seg_start));
        CU(upload(p->seg_block, seg_block));
        CU(upload(p->tile_seg_start, tile_seg_start));
        CU(upload(p->block_seg_start, bss));
        CU(upload(p->block_seg_list, bsl));
        CU(upload(p->tile_order, tord));
    }
    auto& A = p->allocs;
    size_t& B = p->device_bytes;
    {
        std::vector<int32_t> cell(M);
        std::vector<double> fxs(M), fys(M);
        for (int64_t i = 0; i < M; ++i) {
            const int32_t m = order[i];
            cell[i] = (by[m] << 16) | bx[m];
            fxs[i] = frx[m];
            fys[i] = fry[m];
        }
        if (dde) {   // DDE kernels in internal order, for the CSR build below
            const size_t per = (size_t)2 * dde * dde;
            p->h_dde.resize((size_t)M * per);
            for (int64_t i = 0; i < M; ++i)
                std::copy(d->dde_kernels + (size_t)order[i] * per, d->dde_kernels + ((size_t)order[i] + 1) * per,
                          p->h_dde.begin() + (size_t)i * per);
        }
        ALLOC(p->cell, M);
        ALLOC(p->perm, M);
        CU(dalloc_bytes(A, B, &p->fx, M * p->rsz));
        CU(dalloc_bytes(A, B, &p->fy, M * p->rsz));
        CU(upload(p->cell, cell));
        CU(upload(p->perm, order));
        CU(upload_real(p->fx, fxs, p->prec));
        CU(upload_real(p->fy, fys, p->prec));
    }
    {
        std::vector<int32_t> counts = {(int32_t)p->nseg, g.ntiles};
        std::vector<int32_t> ob(p->d, 1), obs(p->b, 1);
        ALLOC(p->counts_all, 2);
        ALLOC(p->ones_block, ob.size());
        ALLOC(p->ones_basis, obs.size());
        CU(upload(p->counts_all, counts));
        CU(upload(p->ones_block, ob));
        CU(upload(p->ones_basis, obs));
    }
    // ---- tables
    {
        CU(dalloc_bytes(A, B, &p->cx, g.nx * p->rsz));
        CU(dalloc_bytes(A, B, &p->cy, g.ny * p->rsz));
        CU(dalloc_bytes(A, B, &p->twx, g.Kx * p->csz));
        CU(dalloc_bytes(A, B, &p->twy, g.Ky * p->csz));
        CU(upload_real(p->cx, deapodisation(g.nx, g.Kx, p->kb_J, g.beta), p->prec));
        CU(upload_real(p->cy, deapodisation(g.ny, g.Ky, p->kb_J, g.beta), p->prec));
        CU(upload_real(p->twx, twiddles(g.Kx), p->prec));
        CU(upload_real(p->twy, twiddles(g.Ky), p->prec));
        {
            std::vector<double> kp = kb_tap_polynomials(p->kb_J, g.beta, KB_DEG);
            for (int a = 0; a < p->kb_J; ++a)
                for (int k = 0; k <= KB_DEG; ++k) p->kbpoly.c[a][k] = (float)kp[(size_t)a * (KB_DEG + 1) + k];
        }
        p->h_filt.assign((size_t)p->b * MAX_FILTER, 0.0);
        p->h_filt_len.assign(p->b, 0);
        for (int k = 0; k < p->b; ++k) {
            const int id = p->basis_ids[k];
            if (id == 0) continue;
            std::vector<double> h = daubechies(id);
            p->h_filt_len[k] = (int)h.size();
            for (size_t j = 0; j < h.size(); ++j) p->h_filt[(size_t)k * MAX_FILTER + j] = h[j];
        }
        CU(dalloc_bytes(A, B, &p->filt, (size_t)p->b * MAX_FILTER * p->rsz));
        ALLOC(p->filt_len, p->b);
        CU(upload_real(p->filt, p->h_filt, p->prec));
        CU(upload(p->filt_len, p->h_filt_len));
    }
    // ---- scratch
    {
        const size_t K = (size_t)g.Kx * g.Ky, N = (size_t)g.nx * g.ny;
        // half-grid intermediates: column panels of the columns 0 .. nx (nx/4 + 1 panels)
        const size_t half_cols = (size_t)(g.nx / 4 + 1) * 4;
        CU(dalloc_bytes(A, B, &p->t1, half_cols * g.ny * p->csz));
        CU(dalloc_bytes(A, B, &p->gridb, half_cols * g.Ky * p->csz));
        CU(cudaMemset(p->t1, 0, half_cols * g.ny * p->csz));
        CU(cudaMemset(p->gridb, 0, half_cols * g.Ky * p->csz));
        CU(dalloc_bytes(A, B, &p->gridu, K * p->csz));
        CU(dalloc_bytes(A, B, &p->rbuf, (size_t)M * p->csz));
        ALLOC(p->seg_part, 2 * std::max<int64_t>(p->nseg, 1));
        ALLOC(p->blk_norm, 2 * p->d);
        CU(dalloc_bytes(A, B, &p->blk_scale, p->d * p->rsz));
        const size_t llsz = (size_t)p->b * (g.ny / 2) * (g.nx / 2) * p->rsz;
        CU(dalloc_bytes(A, B, &p->ll[0], llsz));
        CU(dalloc_bytes(A, B, &p->ll[1], llsz));
        CU(dalloc_bytes(A, B, &p->ds, (size_t)p->b * N * p->rsz));
        CU(dalloc_bytes(A, B, &p->synpart, (size_t)p->b * N * p->rsz));
        p->red_len = 1024;
        ALLOC(p->red, p->red_len + 8);
        ALLOC(p->sched, 8);
        CU(cudaMemset(p->ds, 0, (size_t)p->b * N * p->rsz));
    }
    if (p->g_mode == PD_G_CSR) {
        const size_t nnz = (size_t)g.J * g.J * (size_t)M;
        if (dalloc(A, B, &p->csr_col, nnz) != cudaSuccess ||
            dalloc_bytes(A, B, &p->csr_val, nnz * (p->csr_cplx ? p->csz : p->rsz)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(PD_ENOMEM, "the CSR form of G does not fit in device memory");
        }
        CU(build_csr(p, 0));
        std::vector<double>().swap(p->h_dde);
    }
#undef ALLOC
    CU(cudaDeviceSynchronize());
    return PD_OK;
}

extern "C" pd_status pd_plan_info(const pd_plan* p, int32_t* ky, int32_t* kx, double* beta, int32_t* tile,
                                  int64_t* nsegments, int64_t* ntiles_nonempty, int64_t* device_bytes) {
    if (!p) return fail(PD_EINVAL, "pd_plan_info: null plan");
    if (ky) *ky = p->g.Ky;
    if (kx) *kx = p->g.Kx;
    if (beta) *beta = p->g.beta;
    if (tile) *tile = p->g.tile;
    if (nsegments) *nsegments = p->nseg;
    if (ntiles_nonempty) *ntiles_nonempty = p->ntiles_nonempty;
    if (device_bytes) *device_bytes = (int64_t)p->device_bytes;
    return PD_OK;
}

// ------------------------------------------------------------------ operators
// Scratch of a batch of operator applications (one launch per pass for the whole batch):
// the plan's own buffers for one image, otherwise buffers kept by the plan and grown to
// the largest batch seen (the device is synchronised before the old ones are freed).
static pd_status ensure_batch(pd_plan* p, int batch, void** t1, void** gb, void** gu) {
    if (batch == 1) {
        *t1 = p->t1; *gb = p->gridb; *gu = p->gridu;
        return PD_OK;
    }
    if (batch > p->batch_cap) {
        CU(cudaDeviceSynchronize());
        for (void* q : {p->bt1, p->bgb, p->bgu})
            if (q) {
                cudaFree(q);
                p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), q), p->allocs.end());
            }
        p->bt1 = p->bgb = p->bgu = nullptr;
        p->batch_cap = 0;
        const size_t half = (size_t)(p->g.nx / 4 + 1) * 4;
        size_t dummy = 0;
        if (dalloc_bytes(p->allocs, dummy, &p->bt1, batch * half * p->g.ny * p->csz) ||
            dalloc_bytes(p->allocs, dummy, &p->bgb, batch * half * p->g.Ky * p->csz) ||
            dalloc_bytes(p->allocs, dummy, &p->bgu, (size_t)batch * p->g.Kx * p->g.Ky * p->csz))
            return fail(PD_ENOMEM, "batch scratch allocation failed");
        // the unused slots of the last column panel of the half grids stay zero
        CU(cudaMemset(p->bt1, 0, batch * half * p->g.ny * p->csz));
        CU(cudaMemset(p->bgb, 0, batch * half * p->g.Ky * p->csz));
        p->batch_cap = batch;
    }
    *t1 = p->bt1; *gb = p->bgb; *gu = p->bgu;
    return PD_OK;
}

template <typename R>
static pd_status apply_phi_t(pd_plan* p, const void* x, void* y, int batch, cudaStream_t s) {
    void *t1, *gb, *gu;
    pd_status st = ensure_batch(p, batch, &t1, &gb, &gu);
    if (st != PD_OK) return st;
    CU(fwd_fft<R>(p, (const R*)x, (cplx_t<R>*)gb, s, batch, (cplx_t<R>*)t1));
    CU(degrid_plain<R>(p, (const cplx_t<R>*)gb, (cplx_t<R>*)y, s, batch));
    return PD_OK;
}
template <typename R>
static pd_status apply_phi_adj_t(pd_plan* p, const void* y, void* x, int batch, cudaStream_t s) {
    void *t1, *gb, *gu;
    pd_status st = ensure_batch(p, batch, &t1, &gb, &gu);
    if (st != PD_OK) return st;
    CU(grid_plain<R>(p, (const cplx_t<R>*)y, (cplx_t<R>*)gu, s, batch));
    CU(inv_fft<R>(p, (const cplx_t<R>*)gu, (R*)x, nullptr, s, batch, (cplx_t<R>*)t1));
    return PD_OK;
}

extern "C" pd_status pd_apply_phi(pd_plan* p, const void* x, void* y, int32_t batch, void* stream) {
    if (!p || !x || !y || batch < 1) return fail(PD_EINVAL, "pd_apply_phi: null argument or batch < 1");
    return p->prec == PD_F64 ? apply_phi_t<double>(p, x, y, batch, (cudaStream_t)stream)
                             : apply_phi_t<float>(p, x, y, batch, (cudaStream_t)stream);
}
extern "C" pd_status pd_apply_phi_adj(pd_plan* p, const void* y, void* x, int32_t batch, void* stream) {
    if (!p || !x || !y || batch < 1) return fail(PD_EINVAL, "pd_apply_phi_adj: null argument or batch < 1");
    return p->prec == PD_F64 ? apply_phi_adj_t<double>(p, y, x, batch, (cudaStream_t)stream)
                             : apply_phi_adj_t<float>(p, y, x, batch, (cudaStream_t)stream);
}
extern "C" pd_status pd_apply_psi_adj(pd_plan* p, const void* x, void* coeffs, void* stream) {
    if (!p || !x || !coeffs) return fail(PD_EINVAL, "pd_apply_psi_adj: null argument");
    if (p->prec == PD_F64) CU(psi_adj_plain<double>(p, (const double*)x, (double*)coeffs, (cudaStream_t)stream));
    else CU(psi_adj_plain<float>(p, (const float*)x, (float*)coeffs, (cudaStream_t)stream));
    return PD_OK;
}
extern "C" pd_status pd_apply_psi(pd_plan* p, const void* coeffs, void* x, void* stream) {
    if (!p || !x || !coeffs) return fail(PD_EINVAL, "pd_apply_psi: null argument");
    if (p->prec == PD_F64) CU(psi_plain<double>(p, (const double*)coeffs, (double*)x, (cudaStream_t)stream));
    else CU(psi_plain<float>(p, (const float*)coeffs, (float*)x, (cudaStream_t)stream));
    return PD_OK;
}

extern "C" pd_status pd_sara_weights(pd_plan* p, const void* x, double delta, void* weights, void* stream) {
    if (!p || !x || !weights) return fail(PD_EINVAL, "pd_sara_weights: null argument");
    if (!(delta > 0) || !std::isfinite(delta)) return fail(PD_EINVAL, "pd_sara_weights: delta must be positive and finite");
    if (p->prec == PD_F64) CU(sara_weights<double>(p, (const double*)x, delta, (double*)weights, (cudaStream_t)stream));
    else CU(sara_weights<float>(p, (const float*)x, delta, (float*)weights, (cudaStream_t)stream));
    return PD_OK;
}

// Power method on a symmetric positive operator given as a callback on device images.
template <typename R, typename Op>
static pd_status power_t(pd_plan* p, const R* x0, int max_iter, double tol, R* xa, R* xb, double* dn, Op op,
                         double* lam_out, int* iters, cudaStream_t s) {
    const int64_t N = (int64_t)p->g.nx * p->g.ny;
    double h;
    CU(norm2<R>(p, x0, N, dn, s));
    CU(cudaMemcpyAsync(&h, dn, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (!(h > 0)) return fail(PD_EINVAL, "power method: zero start image");
    CU(scale_copy<R>(x0, xa, N, 1.0 / std::sqrt(h), s));
    double lam = 0.0, prev = 0.0;
    for (int k = 1; k <= max_iter; ++k) {
        pd_status st = op(xa, xb);
        if (st != PD_OK) return st;
        CU(norm2<R>(p, xb, N, dn, s));
        CU(cudaMemcpyAsync(&h, dn, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        lam = std::sqrt(h);
        *iters = k;
        if (lam == 0.0) { *lam_out = 0.0; return PD_OK; }
        CU(scale_copy<R>(xb, xa, N, 1.0 / lam, s));
        if (std::fabs(lam - prev) <= tol * lam) { *lam_out = lam; return PD_OK; }
        prev = lam;
    }
    *lam_out = lam;
    return PD_ENOTCONV;
}

template <typename R>
static pd_status norms_t(pd_plan* p, const void* x0, int max_iter, double tol, double* phi2, double* psi2,
                         int* iters, cudaStream_t s) {
    const int64_t N = (int64_t)p->g.nx * p->g.ny;
    std::vector<void*> tmp;
    size_t bytes = 0;
    R *xa, *xb, *coef;
    cplx_t<R>* vis;
    double* dn;
    auto cleanup = [&]() { free_all(tmp); };
    if (dalloc(tmp, bytes, &xa, N) || dalloc(tmp, bytes, &xb, N) || dalloc(tmp, bytes, &coef, N * p->b) ||
        dalloc(tmp, bytes, &vis, p->M) || dalloc(tmp, bytes, &dn, 1)) {
        cleanup();
        return fail(PD_ENOMEM, "pd_operator_norms: temporary allocation failed");
    }
    int it1 = 0, it2 = 0;
    double l1 = 0, l2 = 0;
    pd_status st1 = power_t<R>(p, (const R*)x0, max_iter, tol, xa, xb, dn,
                               [&](R* a, R* b) {
                                   pd_status q = apply_phi_t<R>(p, a, vis, 1, s);
                                   return q != PD_OK ? q : apply_phi_adj_t<R>(p, vis, b, 1, s);
                               },
                               &l1, &it1, s);
    if (st1 != PD_OK && st1 != PD_ENOTCONV) { cleanup(); return st1; }
    pd_status st2 = power_t<R>(p, (const R*)x0, max_iter, tol, xa, xb, dn,
                               [&](R* a, R* b) {
                                   cudaError_t e = psi_adj_plain<R>(p, a, coef, s);
                                   if (!e) e = psi_plain<R>(p, coef, b, s);
                                   return e ? fail(PD_ECUDA, cudaGetErrorString(e)) : PD_OK;
                               },
                               &l2, &it2, s);
    cleanup();
    if (st2 != PD_OK && st2 != PD_ENOTCONV) return st2;
    if (phi2) *phi2 = l1;
    if (psi2) *psi2 = l2;
    if (iters) *iters = std::max(it1, it2);
    if (st1 == PD_ENOTCONV || st2 == PD_ENOTCONV) return fail(PD_ENOTCONV, "power method: max_iter reached");
    return PD_OK;
}

extern "C" pd_status pd_operator_norms(pd_plan* p, const void* x0, int32_t max_iter, double tol, double* phi_norm2,
                                       double* psi_norm2, int32_t* iterations, void* stream) {
    if (!p || !x0 || max_iter < 1 || !(tol >= 0)) return fail(PD_EINVAL, "pd_operator_norms: bad argument");
    int it = 0;
    pd_status st = p->prec == PD_F64
                       ? norms_t<double>(p, x0, max_iter, tol, phi_norm2, psi_norm2, &it, (cudaStream_t)stream)
                       : norms_t<float>(p, x0, max_iter, tol, phi_norm2, psi_norm2, &it, (cudaStream_t)stream);
    if (iterations) *iterations = it;
    return st;
}

// ------------------------------------------------------------------ state
extern "C" pd_status pd_state_destroy(pd_state* st) {
    if (!st) return PD_OK;
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->ev_in) cudaEventDestroy(st->ev_in);
    if (st->ev_out) cudaEventDestroy(st->ev_out);
    if (st->gstream) cudaStreamDestroy(st->gstream);
    if (st->ev_fork) cudaEventDestroy(st->ev_fork);
    if (st->ev_join) cudaEventDestroy(st->ev_join);
    if (st->pstream) cudaStreamDestroy(st->pstream);
    for (cudaEvent_t e : st->prof_ev)
        if (e) cudaEventDestroy(e);
    free_all(st->allocs);
    delete st;
    return PD_OK;
}

extern "C" pd_status pd_state_create(pd_plan* p, pd_state** out) {
    if (!p || !out) return fail(PD_EINVAL, "pd_state_create: null argument");
    pd_state* st = new pd_state();
    st->plan = p;
    auto& A = st->allocs;
    size_t& B = st->device_bytes;
    const size_t N = (size_t)p->g.nx * p->g.ny, K = (size_t)p->g.Kx * p->g.Ky;
    bool ok = !dalloc_bytes(A, B, &st->x, N * p->rsz) && !dalloc_bytes(A, B, &st->xt, N * p->rsz) &&
              !dalloc_bytes(A, B, &st->s, N * p->b * p->rsz) && !dalloc_bytes(A, B, &st->st, N * p->rsz) &&
              !dalloc_bytes(A, B, &st->v, p->M * p->csz) && !dalloc_bytes(A, B, &st->u, K * p->csz) &&
              !dalloc_bytes(A, B, &st->y, p->M * p->csz) && !dalloc(A, B, &st->eps, p->d) &&
              !dalloc(A, B, &st->res_norm, p->d) && !dalloc(A, B, &st->p_block, p->d) &&
              !dalloc(A, B, &st->p_basis, p->b) && !dalloc(A, B, &st->block_active, p->d) &&
              !dalloc(A, B, &st->basis_active, p->b) &&
              !dalloc(A, B, &st->act_tiles, p->g.ntiles) && !dalloc(A, B, &st->tile_active, p->g.ntiles) &&
              !dalloc(A, B, &st->act_col, p->g.ntiles) && !dalloc(A, B, &st->counts, 6) && !dalloc(A, B, &st->t, 1) && !dalloc(A, B, &st->diag, 2) &&
              !dalloc(A, B, &st->prim_part, 2 * (size_t)inv_rows_ctas(p)) && !dalloc(A, B, &st->status, 1);
    if (!ok) {
        pd_state_destroy(st);
        return fail(PD_ENOMEM, "pd_state_create: device allocation failed");
    }
    for (void* q : A) cudaMemset(q, 0, 16);
    CU(cudaMemset(st->x, 0, N * p->rsz));
    CU(cudaMemset(st->xt, 0, N * p->rsz));
    CU(cudaMemset(st->s, 0, N * p->b * p->rsz));
    CU(cudaMemset(st->st, 0, N * p->rsz));
    CU(cudaMemset(st->v, 0, p->M * p->csz));
    CU(cudaMemset(st->u, 0, K * p->csz));
    CU(cudaMemset(st->y, 0, p->M * p->csz));
    CU(cudaDeviceSynchronize());
    *out = st;
    return PD_OK;
}

extern "C" pd_status pd_state_set_data(pd_plan* p, pd_state* st, const void* y, const double* eps, void* stream) {
    if (!p || !st || !y || !eps || st->plan != p) return fail(PD_EINVAL, "pd_state_set_data: bad argument");
    for (int i = 0; i < p->d; ++i)
        if (!(eps[i] > 0)) return fail(PD_EINVAL, "pd_state_set_data: eps_i must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)p->g.nx * p->g.ny, K = (size_t)p->g.Kx * p->g.Ky;
    if (p->prec == PD_F64) CU(gather_internal<double>(p, (const double2*)y, (double2*)st->y, s));
    else CU(gather_internal<float>(p, (const float2*)y, (float2*)st->y, s));
    CU(cudaMemcpyAsync(st->eps, eps, p->d * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(st->x, 0, N * p->rsz, s));
    CU(cudaMemsetAsync(st->xt, 0, N * p->rsz, s));
    CU(cudaMemsetAsync(st->s, 0, N * p->b * p->rsz, s));
    CU(cudaMemsetAsync(st->st, 0, N * p->rsz, s));
    CU(cudaMemsetAsync(st->v, 0, p->M * p->csz, s));
    CU(cudaMemsetAsync(st->u, 0, K * p->csz, s));
    CU(cudaMemsetAsync(st->t, 0, sizeof(int64_t), s));
    CU(cudaMemsetAsync(st->diag, 0, 2 * sizeof(double), s));
    if (st->syn_at) CU(cudaMemsetAsync(st->syn_at, 0, N * p->b * p->rsz, s));
    if (st->syn_u) CU(cudaMemsetAsync(st->syn_u, 0, N * p->rsz, s));
    std::vector<double> ones_d(p->d, 1.0), ones_b(p->b, 1.0);
    CU(cudaMemcpyAsync(st->p_block, ones_d.data(), p->d * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(st->p_basis, ones_b.data(), p->b * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(init_res_norm(p, st, s));
    CU(cudaStreamSynchronize(s));
    return PD_OK;
}

template <typename R>
static pd_status set_start_t(pd_plan* p, pd_state* st, const void* x0, const void* xt0, const void* s0,
                             const void* v0, cudaStream_t s) {
    const size_t N = (size_t)p->g.nx * p->g.ny, K = (size_t)p->g.Kx * p->g.Ky;
    if (x0) CU(cudaMemcpyAsync(st->x, x0, N * p->rsz, cudaMemcpyDeviceToDevice, s));
    else CU(cudaMemsetAsync(st->x, 0, N * p->rsz, s));
    if (xt0) CU(cudaMemcpyAsync(st->xt, xt0, N * p->rsz, cudaMemcpyDeviceToDevice, s));
    else CU(cudaMemsetAsync(st->xt, 0, N * p->rsz, s));
    if (s0) {
        CU(cudaMemcpyAsync(st->s, s0, N * p->b * p->rsz, cudaMemcpyDeviceToDevice, s));
        CU(psi_plain<R>(p, (const R*)st->s, (R*)st->st, s));                 // s~ = Psi s
    } else {
        CU(cudaMemsetAsync(st->s, 0, N * p->b * p->rsz, s));
        CU(cudaMemsetAsync(st->st, 0, N * p->rsz, s));
    }
    if (v0) {
        CU(gather_internal<R>(p, (const cplx_t<R>*)v0, (cplx_t<R>*)st->v, s));
        CU(grid_plain<R>(p, (const cplx_t<R>*)v0, (cplx_t<R>*)st->u, s));   // U = G^T v
    } else {
        CU(cudaMemsetAsync(st->v, 0, p->M * p->csz, s));
        CU(cudaMemsetAsync(st->u, 0, K * p->csz, s));
    }
    CU(cudaMemsetAsync(st->t, 0, sizeof(int64_t), s));
    CU(cudaMemsetAsync(st->diag, 0, 2 * sizeof(double), s));
    // residual norms of the adaptive probabilities: ||Phi_i x^(0) - y_i||
    if (x0) {
        CU(fwd_fft<R>(p, (const R*)st->x, (cplx_t<R>*)p->gridb, s));
        CU(degrid_res_norms<R>(p, (const cplx_t<R>*)p->gridb, (const cplx_t<R>*)st->y, st->res_norm, s));
    } else {
        CU(init_res_norm(p, st, s));
    }
    CU(cudaStreamSynchronize(s));
    return PD_OK;
}

extern "C" pd_status pd_state_set_start(pd_plan* p, pd_state* st, const void* x0, const void* x_tilde0,
                                        const void* s0, const void* v0, void* stream) {
    if (!p || !st || st->plan != p) return fail(PD_EINVAL, "pd_state_set_start: bad argument");
    return p->prec == PD_F64 ? set_start_t<double>(p, st, x0, x_tilde0, s0, v0, (cudaStream_t)stream)
                             : set_start_t<float>(p, st, x0, x_tilde0, s0, v0, (cudaStream_t)stream);
}

// One iteration of Algorithm 1 on stream s. With `concurrent`, the sparsity-prior
// branch (steps 13-14: reads x~, writes s, s~ and the plan's wavelet scratch) runs on the
// state's second stream between a fork after the draws and a join before the primal
// update, alongside the data-fidelity branch (steps 4-11: FFT, degridding, gridding),
// as step 6 of the algorithm runs its blocks concurrently. Profiled iterations stay on
// one stream so that each kernel phase is timed alone.
static cudaError_t ensure_prior_stream(pd_state* st) {
    if (st->pstream) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&st->pstream, cudaStreamNonBlocking))) return e;
    if ((e = cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming))) return e;
    return cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming);
}

// Steps 3-14 of one iteration: draws, FZx~, degridding and the l2-ball dual update,
// gridding of the dual change into the state's U, and the sparsity dual update with
// s~ (on the second stream when `concurrent`). The join of the two branches is left
// to the caller (enqueue_iteration waits for it before the primal update).
template <typename R>
static cudaError_t enqueue_dual(pd_plan* p, pd_state* st, const pd_params* prm, cudaStream_t s, bool concurrent) {
    cudaError_t e;
    SelectArgs sa{prm->seed, prm->adaptive, prm->adapt_n, prm->adapt_p_min, prm->adapt_p_max};
    if ((e = select_active(p, st, sa, s))) return e;
    cudaStream_t ps = s;
    if (concurrent) {
        if ((e = ensure_prior_stream(st))) return e;
        ps = st->pstream;
        if ((e = cudaEventRecord(st->ev_fork, s))) return e;
        if ((e = cudaStreamWaitEvent(ps, st->ev_fork, 0))) return e;
    }
    if ((e = sparsity_dual<R>(p, (const R*)st->xt, (R*)st->s, (R*)st->st, st->basis_active,
                              prm->kappa * prm->psi_norm, ps, (const R*)prm->sparsity_weights)))
        return e;
    if (concurrent && (e = cudaEventRecord(st->ev_join, ps))) return e;
    if ((e = fwd_fft<R>(p, (const R*)st->xt, (cplx_t<R>*)p->gridb, s))) return e;
    DualArgs da{st->y, st->v, st->block_active, st->eps, st->res_norm};
    if ((e = degrid_dual<R>(p, (const cplx_t<R>*)p->gridb, da, st->act_tiles, st->counts, s))) return e;
    {
        const int q = p->g.ntiles / 4;
        const int32_t* lists[4] = {st->act_col, st->act_col + q, st->act_col + 2 * q, st->act_col + 3 * q};
        if ((e = grid_dual<R>(p, da, lists, st->counts + 2, (cplx_t<R>*)st->u, s))) return e;
    }
    return cudaSuccess;
}

// Steps 17-18 from the gridded dual sum u (the state's own U unless given).
template <typename R>
static cudaError_t enqueue_primal(pd_plan* p, pd_state* st, const pd_params* prm, const void* u, cudaStream_t s) {
    cudaError_t e;
    PrimalArgs pa{prm->tau, prm->sigma, prm->varsigma, st->x, st->xt, st->st, st->prim_part};
    if ((e = inv_fft<R>(p, (const cplx_t<R>*)(u ? u : st->u), nullptr, &pa, s))) return e;
    if ((e = primal_finish(p, st, s))) return e;
    if (prm->adaptive && prm->adapt_exact) {
        // Sec. 4: c_i of the next draw from ||Phi_i x^(t) - y_i|| of every block
        if ((e = fwd_fft<R>(p, (const R*)st->x, (cplx_t<R>*)p->gridb, s))) return e;
        if ((e = degrid_res_norms<R>(p, (const cplx_t<R>*)p->gridb, (const cplx_t<R>*)st->y, st->res_norm, s)))
            return e;
    }
    return cudaSuccess;
}

template <typename R>
static cudaError_t enqueue_iteration(pd_plan* p, pd_state* st, const pd_params* prm, cudaStream_t s,
                                     bool concurrent = true) {
    cudaError_t e;
    if ((e = enqueue_dual<R>(p, st, prm, s, concurrent))) return e;
    if (concurrent && (e = cudaStreamWaitEvent(s, st->ev_join, 0))) return e;
    return enqueue_primal<R>(p, st, prm, nullptr, s);
}

// The plain per-block form of one iteration: the same steps as enqueue_iteration, with
// the active sets drawn on the host (the same counter-based Philox draws) and one launch
// of each data-fidelity operator per active block, one of each sparsity operator per
// active basis. Resources are made on first use.
static cudaError_t ensure_per_block(pd_plan* p, pd_state* st) {
    if (st->pb_eye_blocks) return cudaSuccess;
    const int d = p->d, b = p->b, nt = p->g.ntiles;
    std::vector<int32_t> eyed((size_t)d * d, 0), eyeb((size_t)b * b, 0);
    for (int i = 0; i < d; ++i) eyed[(size_t)i * d + i] = 1;
    for (int j = 0; j < b; ++j) eyeb[(size_t)j * b + j] = 1;
    // each block's tiles, all of them (degridding) and by colour (gridding)
    std::vector<std::vector<int32_t>> tl(d), tc((size_t)4 * d);
    for (int t = 0; t < nt; ++t)
        for (int sg = p->h_tile_seg_start[t]; sg < p->h_tile_seg_start[t + 1]; ++sg) {
            const int blk = p->h_seg_block[sg];
            tl[blk].push_back(t);
            tc[(size_t)4 * blk + tile_colour(t, p->g.ntx)].push_back(t);
        }
    std::vector<int32_t> tiles, counts((size_t)2 * d, 0), col, ccounts((size_t)4 * d, 0);
    st->h_pb_off.assign((size_t)5 * d + 1, 0);   // [d + 1] all-tile offsets, then [4 d] colour offsets
    for (int i = 0; i < d; ++i) {
        st->h_pb_off[i] = (int32_t)tiles.size();
        tiles.insert(tiles.end(), tl[i].begin(), tl[i].end());
        counts[2 * i + 1] = (int32_t)tl[i].size();
        for (int c = 0; c < 4; ++c) {
            st->h_pb_off[d + 1 + 4 * i + c] = (int32_t)col.size();
            col.insert(col.end(), tc[(size_t)4 * i + c].begin(), tc[(size_t)4 * i + c].end());
            ccounts[(size_t)4 * i + c] = (int32_t)tc[(size_t)4 * i + c].size();
        }
    }
    st->h_pb_off[d] = (int32_t)tiles.size();
    cudaError_t e;
    auto& A = st->allocs;
    size_t& B = st->device_bytes;
    if ((e = dalloc(A, B, &st->pb_eye_blocks, eyed.size())) || (e = dalloc(A, B, &st->pb_eye_bases, eyeb.size())) ||
        (e = dalloc(A, B, &st->pb_tiles, std::max<size_t>(tiles.size(), 1))) ||
        (e = dalloc(A, B, &st->pb_counts, counts.size())) ||
        (e = dalloc(A, B, &st->pb_col, std::max<size_t>(col.size(), 1))) ||
        (e = dalloc(A, B, &st->pb_ccounts, ccounts.size())))
        return e;
    if ((e = upload(st->pb_eye_blocks, eyed)) || (e = upload(st->pb_eye_bases, eyeb)) ||
        (e = upload(st->pb_tiles, tiles)) || (e = upload(st->pb_counts, counts)) || (e = upload(st->pb_col, col)) ||
        (e = upload(st->pb_ccounts, ccounts)))
        return e;
    st->h_act.assign(d, 0);
    st->h_actb.assign(b, 0);
    return cudaSuccess;
}

template <typename R>
static cudaError_t enqueue_iteration_per_block(pd_plan* p, pd_state* st, const pd_params* prm, cudaStream_t s) {
    cudaError_t e;
    const int d = p->d, b = p->b;
    const int64_t t = ++st->h_t;
    for (int i = 0; i < d; ++i) st->h_act[i] = philox_uniform(prm->seed, (uint64_t)t, 0, i) < prm->p_block[i];
    for (int j = 0; j < b; ++j) st->h_actb[j] = philox_uniform(prm->seed, (uint64_t)t, 1, j) < prm->p_basis[j];
    // the state's copies of the draws and of t (read by pd_state_report); the host
    // arrays stay untouched until the stream is synchronised at the end of the iteration
    if ((e = cudaMemcpyAsync(st->block_active, st->h_act.data(), d * sizeof(int32_t), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(st->basis_active, st->h_actb.data(), b * sizeof(int32_t), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(st->t, &st->h_t, sizeof(int64_t), cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = fwd_fft<R>(p, (const R*)st->xt, (cplx_t<R>*)p->gridb, s))) return e;
    for (int i = 0; i < d; ++i) {
        if (!st->h_act[i]) continue;
        DualArgs da{st->y, st->v, st->pb_eye_blocks + (size_t)i * d, st->eps, st->res_norm};
        if ((e = degrid_dual<R>(p, (const cplx_t<R>*)p->gridb, da, st->pb_tiles + st->h_pb_off[i],
                                st->pb_counts + 2 * i, s)))
            return e;
    }
    for (int i = 0; i < d; ++i) {
        if (!st->h_act[i]) continue;
        DualArgs da{st->y, st->v, st->pb_eye_blocks + (size_t)i * d, st->eps, st->res_norm};
        const int32_t* lists[4];
        for (int c = 0; c < 4; ++c) lists[c] = st->pb_col + st->h_pb_off[d + 1 + 4 * i + c];
        if ((e = grid_dual<R>(p, da, lists, st->pb_ccounts + 4 * i, (cplx_t<R>*)st->u, s))) return e;
    }
    for (int j = 0; j < b; ++j) {
        if (!st->h_actb[j]) continue;
        if ((e = sparsity_dual<R>(p, (const R*)st->xt, (R*)st->s, (R*)st->st, st->pb_eye_bases + (size_t)j * b,
                                  prm->kappa * prm->psi_norm, s, (const R*)prm->sparsity_weights)))
            return e;
    }
    PrimalArgs pa{prm->tau, prm->sigma, prm->varsigma, st->x, st->xt, st->st, st->prim_part};
    if ((e = inv_fft<R>(p, (const cplx_t<R>*)st->u, nullptr, &pa, s))) return e;
    if ((e = primal_finish(p, st, s))) return e;
    return cudaStreamSynchronize(s);
}

static std::vector<unsigned char> params_key(const pd_plan* p, const pd_params* prm, cudaStream_t s) {
    std::vector<unsigned char> k;
    auto put = [&](const void* src, size_t n) {
        const unsigned char* c = (const unsigned char*)src;
        k.insert(k.end(), c, c + n);
    };
    put(&prm->tau, sizeof(double)); put(&prm->sigma, sizeof(double)); put(&prm->varsigma, sizeof(double));
    put(&prm->kappa, sizeof(double)); put(&prm->psi_norm, sizeof(double)); put(&prm->seed, sizeof(uint64_t));
    put(&prm->adaptive, sizeof(int32_t)); put(&prm->adapt_n, sizeof(double));
    put(&prm->adapt_p_min, sizeof(double)); put(&prm->adapt_p_max, sizeof(double));
    put(&prm->adapt_exact, sizeof(int32_t));
    put(&prm->sparsity_weights, sizeof(void*));
    put(&s, sizeof(s));
    (void)p;
    return k;
}

static pd_status check_params(const pd_plan* p, const pd_params* prm) {
    if (!prm->p_basis || (!prm->adaptive && !prm->p_block)) return fail(PD_EINVAL, "pd_iterate: missing probabilities");
    for (int j = 0; j < p->b; ++j)
        if (!(prm->p_basis[j] > 0 && prm->p_basis[j] <= 1)) return fail(PD_EINVAL, "p_basis must lie in (0, 1]");
    if (!prm->adaptive) {
        for (int i = 0; i < p->d; ++i)
            if (!(prm->p_block[i] > 0 && prm->p_block[i] <= 1)) return fail(PD_EINVAL, "p_block must lie in (0, 1]");
    }
    return PD_OK;
}

extern "C" pd_status pd_iterate_dual(pd_plan* p, pd_state* st, const pd_params* prm, void* stream) {
    if (!p || !st || !prm || st->plan != p) return fail(PD_EINVAL, "pd_iterate_dual: bad argument");
    if (prm->adaptive) return fail(PD_EINVAL, "pd_iterate_dual: adaptive probabilities need every block's residual");
    pd_status q = check_params(p, prm);
    if (q != PD_OK) return q;
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(st->p_block, prm->p_block, p->d * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(st->p_basis, prm->p_basis, p->b * sizeof(double), cudaMemcpyHostToDevice, s));
    if (p->prec == PD_F64) CU(enqueue_dual<double>(p, st, prm, s, true));
    else CU(enqueue_dual<float>(p, st, prm, s, true));
    CU(cudaStreamWaitEvent(s, st->ev_join, 0));
    return PD_OK;
}

extern "C" pd_status pd_iterate_primal(pd_plan* p, pd_state* st, const pd_params* prm, const void* u, void* stream) {
    if (!p || !st || !prm || st->plan != p) return fail(PD_EINVAL, "pd_iterate_primal: bad argument");
    if (prm->adaptive) return fail(PD_EINVAL, "pd_iterate_primal: adaptive probabilities are not split");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->prec == PD_F64) CU(enqueue_primal<double>(p, st, prm, u, s));
    else CU(enqueue_primal<float>(p, st, prm, u, s));
    return PD_OK;
}

extern "C" pd_status pd_state_u(pd_state* st, void** u, int64_t* elements) {
    if (!st || !u) return fail(PD_EINVAL, "pd_state_u: bad argument");
    *u = st->u;
    if (elements) *elements = (int64_t)st->plan->g.Kx * st->plan->g.Ky;
    return PD_OK;
}

// Synthesis form (x = Psi alpha, l1 on the coefficients, positivity as a dual): one
// iteration of the primal-dual template of Algorithm 1 with the roles of the two
// non-smooth terms exchanged. alpha lives in the state's s, x~ in xt; st is scratch.
template <typename R>
static cudaError_t enqueue_synthesis(pd_plan* p, pd_state* st, const pd_params* prm, cudaStream_t s) {
    cudaError_t e;
    SelectArgs sa{prm->seed, 0, 0.0, 0.0, 0.0};
    if ((e = select_active(p, st, sa, s))) return e;                                      // step 3
    if ((e = psi_plain<R>(p, (const R*)st->syn_at, (R*)st->xt, s))) return e;            // x~ = Psi alpha~
    if ((e = fwd_fft<R>(p, (const R*)st->xt, (cplx_t<R>*)p->gridb, s))) return e;        // b~ = F Z x~
    DualArgs da{st->y, st->v, st->block_active, st->eps, st->res_norm};
    if ((e = degrid_dual<R>(p, (const cplx_t<R>*)p->gridb, da, st->act_tiles, st->counts, s))) return e;
    {
        const int q = p->g.ntiles / 4;
        const int32_t* lists[4] = {st->act_col, st->act_col + q, st->act_col + 2 * q, st->act_col + 3 * q};
        if ((e = grid_dual<R>(p, da, lists, st->counts + 2, (cplx_t<R>*)st->u, s))) return e;
    }
    if ((e = inv_fft<R>(p, (const cplx_t<R>*)st->u, (R*)st->st, nullptr, s))) return e;  // Re(Phi^H v)
    if ((e = synth_dual<R>(p, (const R*)st->xt, (R*)st->syn_u, (R*)st->st, prm->sigma, prm->varsigma, s)))
        return e;
    if ((e = psi_adj_plain<R>(p, (const R*)st->st, (R*)p->ds, s))) return e;
    return synth_primal<R>(p, (R*)st->s, (R*)st->syn_at, (const R*)p->ds, prm->tau, prm->tau * prm->kappa, s);
}

extern "C" pd_status pd_synthesis_iterate(pd_plan* p, pd_state* st, const pd_params* prm, int32_t niter,
                                          void* stream) {
    if (!p || !st || !prm || st->plan != p || niter < 0) return fail(PD_EINVAL, "pd_synthesis_iterate: bad argument");
    if (!prm->p_block) return fail(PD_EINVAL, "pd_synthesis_iterate: missing block probabilities");
    if (prm->adaptive || prm->per_block || prm->use_graph || prm->profile)
        return fail(PD_EINVAL, "pd_synthesis_iterate: adaptive, per_block, use_graph and profile must be 0");
    for (int i = 0; i < p->d; ++i)
        if (!(prm->p_block[i] > 0 && prm->p_block[i] <= 1)) return fail(PD_EINVAL, "p_block must lie in (0, 1]");
    if (!(prm->tau > 0)) return fail(PD_EINVAL, "pd_synthesis_iterate: tau must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)p->g.nx * p->g.ny;
    if (!st->syn_at) {
        size_t& B = st->device_bytes;
        if (dalloc_bytes(st->allocs, B, &st->syn_at, N * p->b * p->rsz) ||
            dalloc_bytes(st->allocs, B, &st->syn_u, N * p->rsz)) {
            (void)cudaGetLastError();
            return fail(PD_ENOMEM, "pd_synthesis_iterate: device allocation failed");
        }
        CU(cudaMemsetAsync(st->syn_at, 0, N * p->b * p->rsz, s));
        CU(cudaMemsetAsync(st->syn_u, 0, N * p->rsz, s));
    }
    std::vector<double> ones(p->b, 1.0);   // every basis: the coefficients are primal
    CU(cudaMemcpyAsync(st->p_block, prm->p_block, p->d * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(st->p_basis, ones.data(), p->b * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < niter; ++k) {
        if (p->prec == PD_F64) CU(enqueue_synthesis<double>(p, st, prm, s));
        else CU(enqueue_synthesis<float>(p, st, prm, s));
    }
    // the image x = Psi alpha for pd_state_get_x
    if (p->prec == PD_F64) CU(psi_plain<double>(p, (const double*)st->s, (double*)st->x, s));
    else CU(psi_plain<float>(p, (const float*)st->s, (float*)st->x, s));
    CU(cudaStreamSynchronize(s));   // the host vector of ones is read by the copy above
    return PD_OK;
}

extern "C" pd_status pd_iterate(pd_plan* p, pd_state* st, const pd_params* prm, int32_t niter, void* stream) {
    if (!p || !st || !prm || st->plan != p || niter < 0) return fail(PD_EINVAL, "pd_iterate: bad argument");
    if (!prm->p_basis || (!prm->adaptive && !prm->p_block)) return fail(PD_EINVAL, "pd_iterate: missing probabilities");
    for (int j = 0; j < p->b; ++j)
        if (!(prm->p_basis[j] > 0 && prm->p_basis[j] <= 1)) return fail(PD_EINVAL, "p_basis must lie in (0, 1]");
    if (!prm->adaptive) {
        for (int i = 0; i < p->d; ++i)
            if (!(prm->p_block[i] > 0 && prm->p_block[i] <= 1)) return fail(PD_EINVAL, "p_block must lie in (0, 1]");
    } else {
        const double nd = prm->adapt_n / p->d;
        if (!(prm->adapt_n > 0 && prm->adapt_n <= p->d && prm->adapt_p_min >= 0 && prm->adapt_p_min <= nd &&
              prm->adapt_p_min <= prm->adapt_p_max && prm->adapt_p_max <= 1 && prm->adapt_p_max >= nd))
            return fail(PD_EINVAL, "adaptive probabilities need 0 <= p_min <= n/d <= p_max <= 1");
    }
    if (prm->per_block && (prm->adaptive || prm->use_graph || prm->profile))
        return fail(PD_EINVAL, "pd_iterate: the per-block form needs adaptive = 0, use_graph = 0 and profile = 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (!prm->adaptive) CU(cudaMemcpyAsync(st->p_block, prm->p_block, p->d * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(st->p_basis, prm->p_basis, p->b * sizeof(double), cudaMemcpyHostToDevice, s));
    if (niter == 0) return PD_OK;
    if (prm->per_block) {
        CU(ensure_per_block(p, st));
        CU(cudaMemcpyAsync(&st->h_t, st->t, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (int k = 0; k < niter; ++k) {
            if (p->prec == PD_F64) CU(enqueue_iteration_per_block<double>(p, st, prm, s));
            else CU(enqueue_iteration_per_block<float>(p, st, prm, s));
        }
        return PD_OK;
    }
    if (prm->use_graph) {
        // The caller's stream may be the legacy default stream, which cannot be captured:
        // capture and replay on the state's private stream, fenced by events both ways.
        if (!st->gstream) {
            CU(cudaStreamCreateWithFlags(&st->gstream, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&st->ev_in, cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming));
        }
        cudaStream_t gs = st->gstream;
        CU(cudaEventRecord(st->ev_in, s));
        CU(cudaStreamWaitEvent(gs, st->ev_in, 0));
        std::vector<unsigned char> key = params_key(p, prm, gs);
        if (!st->gexec || key != st->gkey) {
            if (st->gexec) { cudaGraphExecDestroy(st->gexec); st->gexec = nullptr; }
            // relaxed mode: kernel attribute calls made while enqueueing are allowed
            CU(cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed));
            cudaError_t e = p->prec == PD_F64 ? enqueue_iteration<double>(p, st, prm, gs)
                                              : enqueue_iteration<float>(p, st, prm, gs);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(gs, &graph);
            if (e) { if (graph) cudaGraphDestroy(graph); return fail(PD_ECUDA, std::string("capture: ") + cudaGetErrorString(e)); }
            CU(e2);
            cudaError_t e3 = cudaGraphInstantiate(&st->gexec, graph, 0);
            cudaGraphDestroy(graph);
            CU(e3);
            st->gkey = key;
        }
        for (int k = 0; k < niter; ++k) CU(cudaGraphLaunch(st->gexec, gs));
        CU(cudaEventRecord(st->ev_out, gs));
        CU(cudaStreamWaitEvent(s, st->ev_out, 0));
    } else if (prm->profile) {
        if (!st->prof_ev[0])
            for (cudaEvent_t& e : st->prof_ev) CU(cudaEventCreate(&e));
        for (int k = 0; k < niter; ++k) {
            for (cudaEvent_t e : st->prof_ev) CU(cudaEventRecord(e, s));   // phases not run read 0 ms
            g_prof = st;
            cudaError_t e = p->prec == PD_F64 ? enqueue_iteration<double>(p, st, prm, s, false)
                                              : enqueue_iteration<float>(p, st, prm, s, false);
            g_prof = nullptr;
            CU(e);
            CU(cudaStreamSynchronize(s));
            for (int ph = 0; ph < PH_COUNT; ++ph) {
                float ms = 0.f;
                CU(cudaEventElapsedTime(&ms, st->prof_ev[2 * ph], st->prof_ev[2 * ph + 1]));
                st->prof_ms[ph] += ms;
                st->prof_n[ph] += 1;
            }
        }
    } else {
        for (int k = 0; k < niter; ++k) {
            if (p->prec == PD_F64) CU(enqueue_iteration<double>(p, st, prm, s));
            else CU(enqueue_iteration<float>(p, st, prm, s));
        }
    }
    return PD_OK;
}

extern "C" pd_status pd_state_profile(pd_state* st, double* ms, int64_t* iterations, int32_t n, int32_t reset) {
    if (!st || n < 0) return fail(PD_EINVAL, "pd_state_profile: bad argument");
    for (int ph = 0; ph < PH_COUNT && ph < n; ++ph) {
        if (ms) ms[ph] = st->prof_ms[ph];
        if (iterations) iterations[ph] = st->prof_n[ph];
    }
    if (reset)
        for (int ph = 0; ph < PH_COUNT; ++ph) { st->prof_ms[ph] = 0.0; st->prof_n[ph] = 0; }
    return PD_OK;
}

extern "C" pd_status pd_state_get_x(const pd_state* st, void* x, void* stream) {
    if (!st || !x) return fail(PD_EINVAL, "pd_state_get_x: null argument");
    const pd_plan* p = st->plan;
    CU(cudaMemcpyAsync(x, st->x, (size_t)p->g.nx * p->g.ny * p->rsz, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PD_OK;
}
extern "C" pd_status pd_state_get_x_tilde(const pd_state* st, void* x, void* stream) {
    if (!st || !x) return fail(PD_EINVAL, "pd_state_get_x_tilde: null argument");
    const pd_plan* p = st->plan;
    CU(cudaMemcpyAsync(x, st->xt, (size_t)p->g.nx * p->g.ny * p->rsz, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PD_OK;
}
extern "C" pd_status pd_state_get_s(const pd_state* st, void* s, void* stream) {
    if (!st || !s) return fail(PD_EINVAL, "pd_state_get_s: null argument");
    const pd_plan* p = st->plan;
    CU(cudaMemcpyAsync(s, st->s, (size_t)p->b * p->g.nx * p->g.ny * p->rsz, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return PD_OK;
}
extern "C" pd_status pd_state_get_v(const pd_plan* p, const pd_state* st, void* v, void* stream) {
    if (!p || !st || !v || st->plan != p) return fail(PD_EINVAL, "pd_state_get_v: bad argument");
    if (p->prec == PD_F64) CU(scatter_user<double>(p, (const double2*)st->v, (double2*)v, (cudaStream_t)stream));
    else CU(scatter_user<float>(p, (const float2*)st->v, (float2*)v, (cudaStream_t)stream));
    return PD_OK;
}

extern "C" pd_status pd_state_report(const pd_plan* p, const pd_state* st, int64_t* t, double* dx2, double* x2,
                                     double* res_norm, double* p_block, int32_t* block_active, int32_t* basis_active,
                                     int32_t* work, void* stream) {
    if (!p || !st || st->plan != p) return fail(PD_EINVAL, "pd_state_report: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t th = 0;
    double dg[2] = {0, 0};
    CU(cudaMemcpyAsync(&th, st->t, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(dg, st->diag, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (res_norm) CU(cudaMemcpyAsync(res_norm, st->res_norm, p->d * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (p_block) CU(cudaMemcpyAsync(p_block, st->p_block, p->d * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (block_active) CU(cudaMemcpyAsync(block_active, st->block_active, p->d * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (basis_active) CU(cudaMemcpyAsync(basis_active, st->basis_active, p->b * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (work) CU(cudaMemcpyAsync(work, st->counts, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (t) *t = th;
    if (dx2) *dx2 = dg[0];
    if (x2) *x2 = dg[1];
    return PD_OK;
}

// checkpoint layout: x, xt, s, st, v, u, y (working precision), eps, res_norm, p_block, p_basis, t
struct Part { void* dev; size_t bytes; };
static std::vector<Part> state_parts(const pd_plan* p, const pd_state* st) {
    const size_t N = (size_t)p->g.nx * p->g.ny, K = (size_t)p->g.Kx * p->g.Ky;
    return {{st->x, N * p->rsz}, {st->xt, N * p->rsz}, {st->s, N * p->b * p->rsz}, {st->st, N * p->rsz},
            {st->v, p->M * p->csz}, {st->u, K * p->csz}, {st->y, p->M * p->csz}, {st->eps, p->d * sizeof(double)},
            {st->res_norm, p->d * sizeof(double)}, {st->p_block, p->d * sizeof(double)},
            {st->p_basis, p->b * sizeof(double)}, {st->t, sizeof(int64_t)}};
}
extern "C" size_t pd_state_bytes(const pd_plan* p) {
    if (!p) return 0;
    pd_state dummy;
    size_t n = 0;
    for (const Part& q : state_parts(p, &dummy)) n += q.bytes;
    return n;
}
extern "C" pd_status pd_state_save(const pd_plan* p, const pd_state* st, void* buf, void* stream) {
    if (!p || !st || !buf || st->plan != p) return fail(PD_EINVAL, "pd_state_save: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* c = (unsigned char*)buf;
    for (const Part& q : state_parts(p, st)) {
        CU(cudaMemcpyAsync(c, q.dev, q.bytes, cudaMemcpyDeviceToHost, s));
        c += q.bytes;
    }
    CU(cudaStreamSynchronize(s));
    return PD_OK;
}
extern "C" pd_status pd_state_load(const pd_plan* p, pd_state* st, const void* buf, void* stream) {
    if (!p || !st || !buf || st->plan != p) return fail(PD_EINVAL, "pd_state_load: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char* c = (const unsigned char*)buf;
    for (const Part& q : state_parts(p, st)) {
        CU(cudaMemcpyAsync(q.dev, c, q.bytes, cudaMemcpyHostToDevice, s));
        c += q.bytes;
    }
    CU(cudaStreamSynchronize(s));
    return PD_OK;
}

extern "C" pd_status pd_plan_autotune(const pd_plan_desc* desc, const int32_t* candidates, int32_t ncand,
                                      int32_t iters, int32_t* best_tile, double* ms, void* stream) {
    if (!desc || !candidates || ncand < 1 || iters < 1 || !best_tile)
        return fail(PD_EINVAL, "pd_plan_autotune: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    double best = -1.0;
    *best_tile = 0;
    for (int k = 0; k < ncand; ++k) {
        if (ms) ms[k] = -1.0;
        pd_plan_desc d = *desc;
        d.tile = candidates[k];
        pd_plan* p = nullptr;
        if (pd_plan_create(&d, &p) != PD_OK) continue;
        pd_state* st = nullptr;
        pd_status rc = pd_state_create(p, &st);
        void* y = nullptr;
        if (rc == PD_OK && cudaMalloc(&y, (size_t)p->M * p->csz) != cudaSuccess) rc = PD_ENOMEM;
        double t_ms = -1.0;
        if (rc == PD_OK) {
            cudaMemsetAsync(y, 0, (size_t)p->M * p->csz, s);
            std::vector<double> eps(p->d, 1.0), pb(p->d, 0.5), pbs(p->b, 0.5);
            pd_params prm{};
            prm.tau = 0.49; prm.sigma = 1.0; prm.varsigma = 1e-3; prm.kappa = 1e-3; prm.psi_norm = 1.0;
            prm.seed = 1; prm.p_block = pb.data(); prm.p_basis = pbs.data(); prm.use_graph = 1;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (pd_state_set_data(p, st, y, eps.data(), stream) == PD_OK &&
                pd_iterate(p, st, &prm, 1, stream) == PD_OK && cudaEventCreate(&e0) == cudaSuccess &&
                cudaEventCreate(&e1) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess &&
                pd_iterate(p, st, &prm, iters, stream) == PD_OK && cudaEventRecord(e1, s) == cudaSuccess &&
                cudaEventSynchronize(e1) == cudaSuccess) {
                float f = 0.f;
                if (cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) t_ms = f / iters;
            }
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
        if (y) cudaFree(y);
        pd_state_destroy(st);
        pd_plan_destroy(p);
        if (ms) ms[k] = t_ms;
        if (t_ms > 0 && (best < 0 || t_ms < best)) { best = t_ms; *best_tile = candidates[k]; }
    }
    if (*best_tile == 0) return fail(PD_EINVAL, "pd_plan_autotune: no candidate tile could be planned and run");
    return PD_OK;
}
