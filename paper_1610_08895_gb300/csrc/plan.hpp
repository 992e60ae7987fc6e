// Internal plan/state layout of the PD-R CUDA library and the launcher interfaces
// between the host API (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "pd.h"

namespace pdgb {

constexpr int PW = 4;          // panel width (complex elements) of the column-panel grid layout
constexpr int MAX_FILTER = 16; // longest Daubechies filter (db8)
constexpr int MAX_BASES = 16;

// Device-side view of the plan, passed by value to kernels.
struct Geo {
    int nx, ny, Kx, Ky;
    int J;
    double beta;
    int tile, logT, ntx, nty, ntiles;
    int ext;        // T + J - 1: extended tile edge of the gridding accumulator
    int halo_lo;    // J/2 - 1 cells before the tile
    int halo_hi;    // J/2 cells after the tile
};

// Tile colour classes of the gridding: (tile row parity, tile column parity). Two tiles
// of one colour are at least two tiles apart, so for J - 1 <= T their windows (tile plus
// halo) are disjoint and one launch may update them in U without atomics. The grid has
// at least two tiles per side (an even number), so the four classes are equal in size.
__host__ __device__ __forceinline__ int tile_colour(int t, int ntx) { return (((t / ntx) & 1) << 1) | ((t % ntx) & 1); }

// Monomial coefficients (in x = 2 f - 1) of the per-tap Chebyshev interpolants of the
// Kaiser-Bessel weight phi(f + J/2 - 1 - a), used by the FP32 kernels.
constexpr int KB_DEG = 10;
struct KbPoly {
    float c[16][KB_DEG + 1];
};

// Super-cells of SC x SC base cells inside a tile: the visibilities of a segment are
// sorted by super-cell, then row-major by base cell (the gridding's super-rows).
constexpr int SC = 8;

// Element offset of grid cell (ky, kx) in the column-panel layout [Kx/PW][K][PW].
__host__ __device__ __forceinline__ int64_t panel_off(int ky, int kx, int K) {
    return ((int64_t)(kx >> 2) * K + ky) * PW + (kx & 3);
}

}  // namespace pdgb

struct pd_plan {
    int prec;                  // PD_F32 / PD_F64
    size_t rsz, csz;           // sizeof real / complex
    pdgb::Geo g;
    int64_t M;
    int d, b, L;
    std::vector<int> basis_ids;
    int n_wavelet;             // bases with id > 0
    int64_t nseg;
    int ntiles_nonempty;
    int num_sms;
    int device;

    // host copies of the static tables
    std::vector<int32_t> h_tile_seg_start, h_seg_block, h_block_seg_start, h_block_seg_list;

    // device: visibilities in internal (tile, block, row, column) order
    int32_t* cell = nullptr;       // (by << 16) | bx of floor(g), mod K
    void* fx = nullptr;            // real [M]: fractional part of g_x
    void* fy = nullptr;
    int32_t* perm = nullptr;       // internal -> user index
    int g_mode = PD_G_ON_THE_FLY;  // PD_G_CSR: G stored explicitly, below
    int kb_J = 0;                  // interpolation kernel width (g.J is the footprint: kb_J + dde - 1)
    int dde = 0;                   // DDE kernel width d (0: none)
    bool csr_cplx = false;         // CSR entries complex (DDE-aware G)
    std::vector<double> h_dde;     // DDE kernels, internal order (kept until G is built)
    int32_t* csr_col = nullptr;    // [J^2][M] grid cell (ky << 16 | kx) of each entry, internal order
    void* csr_val = nullptr;       // real [J^2][M] weight of each entry
    int32_t* seg_start = nullptr;  // [nseg + 1]
    int32_t* seg_block = nullptr;  // [nseg]
    int32_t* tile_seg_start = nullptr;  // [ntiles + 1]
    int nsc_side = 0;                      // super-cells per tile side (tile / SC)
    int32_t* seg_sc_start = nullptr;       // [nseg][nsc_side^2 + 1] super-cell starts inside each segment
    std::vector<int32_t> h_sc_start;       // (host, only during plan construction)
    int max_tile_segs = 0;                 // most (tile, block) segments in one tile
    pdgb::KbPoly kbpoly{};
    int32_t* block_seg_start = nullptr;    // [d + 1] into block_seg_list
    int32_t* block_seg_list = nullptr;     // [nseg] segments of each block, tile order
    int32_t* tile_order = nullptr;         // [ntiles] tiles by decreasing visibility count
    int32_t* colour_tiles = nullptr;       // [4][ntiles/4] tiles of each colour, heaviest first
    int32_t* colour_counts = nullptr;      // [4] ntiles/4 each
    int32_t* counts_all = nullptr;         // {nseg, ntiles}
    int32_t* ones_block = nullptr;         // all blocks active
    int32_t* ones_basis = nullptr;

    // tables
    void* cx = nullptr;            // real [nx] deapodisation
    void* cy = nullptr;            // real [ny]
    void* twx = nullptr;           // complex [Kx]: exp(-2 pi i k / Kx)
    void* twy = nullptr;           // complex [Ky]
    void* filt = nullptr;          // real [b][MAX_FILTER] low-pass filters (0 for Dirac)
    int32_t* filt_len = nullptr;   // [b]
    std::vector<double> h_filt;    // host copy
    std::vector<int> h_filt_len;

    // scratch
    void* t1 = nullptr;            // complex [nx/PW + 1][ny][PW] half-spectrum row-pass intermediate
    void* gridb = nullptr;         // complex [nx/PW + 1][Ky][PW] b~ = F Z x~, columns 0 .. nx
    void* gridu = nullptr;         // complex grid for the plain adjoint
    int batch_cap = 0;             // images the batch scratch below holds (0: none yet)
    void* bt1 = nullptr;           // batch scratch of pd_apply_phi / pd_apply_phi_adj: t1, F Z x, U
    void* bgb = nullptr;
    void* bgu = nullptr;
    void* rbuf = nullptr;          // complex [M] residuals r = v + G b - y (internal order)
    double* seg_part = nullptr;    // [2 * nseg] per-segment FP64 partial norms
    double* blk_norm = nullptr;    // [2 * d]: ||r_i||^2, ||G_i b - y_i||^2
    void* blk_scale = nullptr;     // real [d]: max(0, 1 - eps_i / ||r_i||)
    void* ll[2] = {nullptr, nullptr};  // real [b][ny/2][nx/2] wavelet approximation ping-pong
    void* ds = nullptr;            // real [b][ny][nx] change of the sparsity duals
    void* synpart = nullptr;       // real [b][ny][nx] level-0 synthesis of each basis
    double* red = nullptr;         // reduction scratch
    int32_t* sched = nullptr;      // [8] work counters of the dynamically scheduled launches (0-3 gridding
                                   // colours, 4 degridding)
    int red_len = 0;
    size_t device_bytes = 0;
    std::vector<void*> allocs;     // every device allocation of the plan
};

struct pd_state {
    pd_plan* plan = nullptr;
    void* x = nullptr;
    void* xt = nullptr;
    void* s = nullptr;             // [b][ny][nx]
    void* st = nullptr;            // s~ = Psi s
    void* syn_at = nullptr;        // synthesis form: alpha~ [b][ny][nx] (alpha lives in s)
    void* syn_u = nullptr;         // synthesis form: positivity dual u [ny][nx]
    void* v = nullptr;             // complex [M] internal order
    void* u = nullptr;             // complex grid G^T v (panel layout)
    void* y = nullptr;             // complex [M] internal order
    double* eps = nullptr;         // [d]
    double* res_norm = nullptr;    // [d]
    double* p_block = nullptr;     // [d]
    double* p_basis = nullptr;     // [b]
    int32_t* block_active = nullptr;   // [d]
    int32_t* basis_active = nullptr;   // [b]
    int32_t* act_tiles = nullptr;      // [ntiles] tiles holding an active block, heaviest first
    int32_t* act_col = nullptr;        // [4][ntiles/4] the same tiles split by colour
    int32_t* tile_active = nullptr;    // [ntiles]: tile holds a visibility of an active block
    int32_t* counts = nullptr;         // {active segments, active tiles, active tiles of colour 0..3}
    int64_t* t = nullptr;              // iteration counter (device)
    double* diag = nullptr;            // [2]: ||dx||^2, ||x||^2
    double* prim_part = nullptr;       // [2 * ny / rows-per-CTA]
    int32_t* status = nullptr;         // device status word
    std::vector<void*> allocs;
    size_t device_bytes = 0;
    // CUDA graph of one iteration
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    cudaStream_t gstream = nullptr;    // private stream the graph is captured on and replayed on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // second stream for the sparsity-prior branch of an iteration (Alg. 1 steps 12-15
    // run concurrently with the data-fidelity steps 6-11), with its fork/join events
    cudaStream_t pstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // plain per-block form (pd_params.per_block): one-hot activity flags, each block's tiles
    int32_t* pb_eye_blocks = nullptr;  // [d][d]
    int32_t* pb_eye_bases = nullptr;   // [b][b]
    int32_t* pb_tiles = nullptr;       // tiles of block i at pb_tiles[h_pb_off[i] ...]
    int32_t* pb_counts = nullptr;      // [d][2]: {0, number of tiles of block i}
    int32_t* pb_col = nullptr;         // tiles of block i and colour c at pb_col[h_pb_off[4 i + c] ...]
    int32_t* pb_ccounts = nullptr;     // [d][4] number of tiles of block i per colour
    std::vector<int32_t> h_pb_off;
    std::vector<int32_t> h_act, h_actb;
    int64_t h_t = 0;
    // per-phase timing (pd_params.profile)
    cudaEvent_t prof_ev[2 * 12] = {};
    double prof_ms[12] = {};
    int64_t prof_n[12] = {};
};

namespace pdgb {

// Kernel phases of one iteration, for optional per-phase CUDA-event timing.
enum Phase {
    PH_SELECT = 0, PH_FWD_ROWS, PH_FWD_COLS, PH_DEGRID, PH_NORMS, PH_GRID, PH_ANALYSIS,
    PH_SYNTHESIS, PH_INV_COLS, PH_INV_ROWS, PH_FINISH, PH_COUNT
};
// Record the start (end = 0) or end (end = 1) event of a phase on stream s when the
// calling thread has profiling switched on; otherwise a no-op.
void prof_mark(int phase, int end, cudaStream_t s);
// Record `msg` as the calling thread's last error (pd_last_error) and return `st`.
pd_status set_error(pd_status st, const char* msg);

// ---- fft.cu
// batch images at once (blockIdx.y); t1: the half-spectrum intermediate of the batch
// (nullptr = the plan's own, for batch 1)
template <typename R>
cudaError_t fwd_fft(const pd_plan* p, const R* x, cplx_t<R>* grid, cudaStream_t s, int batch = 1,
                    cplx_t<R>* t1 = nullptr);
struct PrimalArgs {
    double tau, sigma, varsigma;
    void* x;           // in/out
    void* xt;          // out
    const void* st;    // s~
    double* part;      // per-CTA partial sums
};
// mode 0: write Re(Z^T F^H grid) to out; mode 1: primal update (Alg. 1 steps 17-18)
template <typename R>
cudaError_t inv_fft(const pd_plan* p, const cplx_t<R>* grid, R* out, const PrimalArgs* pa, cudaStream_t s,
                    int batch = 1, cplx_t<R>* t1 = nullptr);
int inv_rows_ctas(const pd_plan* p);

// ---- gridding.cu
struct DualArgs {
    const void* y;        // internal-order data (pd mode) or user-order input (plain mode)
    void* v;              // dual (pd mode)
    const int32_t* block_active;
    const double* eps;
    double* res_norm;     // updated for active blocks
};
// plain degrid of `batch` half grids (stride: one image's half grid) into out (user order, stride M)
template <typename R>
cudaError_t degrid_plain(const pd_plan* p, const cplx_t<R>* grid, cplx_t<R>* out_user, cudaStream_t s, int batch = 1);
// ||G_i grid - y_i|| of every block into res_norm (the exact reading of Sec. 4's c_i)
template <typename R>
cudaError_t degrid_res_norms(const pd_plan* p, const cplx_t<R>* grid, const cplx_t<R>* y, double* res_norm,
                             cudaStream_t s);
// pd degrid over the listed tiles: r = v + G b - y, segment partial norms, then block scales
template <typename R>
cudaError_t degrid_dual(const pd_plan* p, const cplx_t<R>* grid, const DualArgs& a, const int32_t* tiles,
                        const int32_t* counts, cudaStream_t s);
// G in CSR form (PD_G_CSR): the J^2 (cell, weight) entries of every visibility
cudaError_t build_csr(pd_plan* p, cudaStream_t s);
// plain grid: U = G^T y_user (U overwritten) for `batch` inputs (stride M) and grids (stride Kx Ky)
template <typename R>
cudaError_t grid_plain(const pd_plan* p, const cplx_t<R>* y_user, cplx_t<R>* U, cudaStream_t s, int batch = 1);
// pd grid over the listed tiles, one launch per colour (tiles[c]: device list of colour c,
// counts4[c]: device count): v <- scale * r, U += G^T (v_new - v_old)
template <typename R>
cudaError_t grid_dual(const pd_plan* p, const DualArgs& a, const int32_t* const* tiles, const int32_t* counts4,
                      cplx_t<R>* U, cudaStream_t s);

// ---- wavelet.cu
// plain analysis: coeffs[b][ny][nx] = Psi^H x
template <typename R>
cudaError_t psi_adj_plain(const pd_plan* p, const R* x, R* coeffs, cudaStream_t s);
// plain synthesis: x = Psi coeffs
template <typename R>
cudaError_t psi_plain(const pd_plan* p, const R* coeffs, R* x, cudaStream_t s);
// pd: for active bases s <- clip(s + Psi_j^H x~ / sqrt(b), -alpha, alpha); s~ += Psi (s_new - s_old)
template <typename R>
cudaError_t sparsity_dual(const pd_plan* p, const R* xt, R* s, R* st, const int32_t* basis_active,
                          double alpha, cudaStream_t s_, const R* wt = nullptr);
// weights of the reweighted prior: w = delta / (delta + |Psi^H x|), w real [b][ny][nx]
template <typename R>
cudaError_t sara_weights(const pd_plan* p, const R* x, double delta, R* w, cudaStream_t s);

// ---- pd_kernels.cu
struct SelectArgs {
    uint64_t seed;
    int adaptive;
    double n, p_min, p_max;
};
cudaError_t select_active(const pd_plan* p, pd_state* st, const SelectArgs& a, cudaStream_t s);
// synthesis form: positivity dual and image-domain primal term; primal step on the coefficients
template <typename R>
cudaError_t synth_dual(const pd_plan* p, const R* xt, R* u, R* back, double sigma, double varsigma, cudaStream_t s);
template <typename R>
cudaError_t synth_primal(const pd_plan* p, R* alpha, R* alpha_t, const R* w, double tau, double thr, cudaStream_t s);
cudaError_t primal_finish(const pd_plan* p, pd_state* st, cudaStream_t s);
template <typename R>
cudaError_t norm2(const pd_plan* p, const R* x, int64_t n, double* out, cudaStream_t s);
template <typename R>
cudaError_t scale_copy(const R* x, R* y, int64_t n, double scale, cudaStream_t s);
template <typename R>
cudaError_t gather_internal(const pd_plan* p, const cplx_t<R>* user, cplx_t<R>* internal, cudaStream_t s);
template <typename R>
cudaError_t scatter_user(const pd_plan* p, const cplx_t<R>* internal, cplx_t<R>* user, cudaStream_t s);
cudaError_t init_res_norm(const pd_plan* p, pd_state* st, cudaStream_t s);

}  // namespace pdgb
