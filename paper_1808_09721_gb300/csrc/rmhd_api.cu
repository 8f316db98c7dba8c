// rmhd_api.cu -- C ABI of the library (declared in include/rmhd.h): context
// and workspace management, host <-> device transfers, and the SSP2(222)
// IMEX step sequence (Sec. 2.2.1 and Table 1 of Wright & Hawke,
// arXiv:1808.09721):
//
//   stage 1:  q1 = q^n + g dt Psi(q1)                         (per-cell solve)
//   flux 1:   r2 = q^n + dt L(q1) + (1 - 2g) dt Psi(q1),
//             acc = q^n + dt/2 (L(q1) + Psi(q1))               (fused)
//   stage 2:  q2 = r2 + g dt Psi(q2)                           (per-cell solve)
//   flux 2:   q^{n+1} = acc + dt/2 (L(q2) + Psi(q2)), w^{n+1} = recovery   (fused)
//
// with g = 1 - 1/sqrt(2). One step is captured once in a CUDA graph per time
// step size and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rmhd.h"
#include "rmhd_internal.h"

using namespace rmhd;

struct rmhd_ctx {
    rmhd_config cfg;
    Grid g;
    Phys ph;
    cudaStream_t stream;
    int device;
    bool own_ws;
    char *ws;
    size_t ws_bytes;
    double *Q, *W, *Q1, *W1, *R, *ACC, *stage_buf, *scratch, *diag;
    double *R3;    // SSP3(332): q^n + dt/4 L1 + (1/2 - gamma) dt Psi1 (null for SSP2)
    double *LBUF;  // 3-D grids: L_x + L_y of the current flux pass (null otherwise)
    double *SRCG;  // planes handed from the FP64 stage kernel to the line-sweep flux pass (null in batches)
    int *status;       // device [2]
    unsigned long long *hist;  // device [44]: solver statistics (FP32 iterations, FP64 passes, starts)
    int *rlist;                // device [2 + rcap]: cells whose first stage-solve start failed
    int rcap;
    int first_start;           // rmhd_set_first_start (tests of the restart path)
    bool stats_on;             // count stage solves into hist
    int maxpass;               // cap on the FP64 refinement passes (0: the kernels' default)
    int *h_status;     // pinned host copy of the 64-bit status key
    double *h_diag;    // pinned host [8]
    bool has_state;
    bool fresh_prims;  // state set by rmhd_set_prims and not stepped since
    bool w_stale;      // W holds a warm start (stage-2 primitives), not the primitives of Q
    double t;
    cudaGraphExec_t graph;
    double graph_dt;
    bool profiling;
    // batched ensemble of 1-D runs (batch == true)
    bool batch;
    int nruns, nwork;
    std::vector<int> run_nx;
    std::vector<long long> run_off;
    std::vector<double> run_dx, run_sigma;
    BatchArgs bargs;
    int *d_nx, *d_run_of;
    int2 *d_work;
    long long *d_off;
    double *d_dx, *d_rdx4, *d_dt, *d_sigma, *d_eta, *d_adt, *d_cpsi;
    double *h_tab;       // pinned host staging for the per-run time-step tables
    double *Qsave, *Wsave;
    int tile_x, flux_blocks, stage_threads;
    double tab_dt;       // dt the tables were built for (<= 0: per-run CFL)
    // recording for the discrete adjoint
    bool recording;
    int rec_nsteps, rec_K, rec_done;
    double rec_dt;
    char *rec_ws;
    bool rec_own;
    double *rec_ck, *rec_seg, *rec_lam, *rec_lamn, *rec_lq, *rec_lr2, *rec_lr3, *rec_fx, *rec_fy, *rec_fz, *rec_fbx,
        *rec_fby, *rec_fbz,
        *rec_qbd, *rec_sig, *rec_pbar, *rec_fin, *rec_sum;
    // slab of a domain decomposed along y (rmhd_create_slab)
    bool slab;
    int slab_j0, slab_ny;   // first global row, global rows
    double *HLO, *HHI;      // halo rows below / above ([NC + NW][2][nx] each)
    // phase-by-phase stepping (rmhd_step_phase)
    int phase_next;         // next phase of the current step (0: between steps)
    double phase_dt;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::string err;
};

static const double kGamma = 1.0 - 0.70710678118654752440;  // 1 - 1/sqrt(2)

static int fail(rmhd_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
static int fail(rmhd_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK(c, call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail((c), RMHD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int validate(const rmhd_config *cfg) {
    if (!cfg) return RMHD_ERR_INVALID;
    if (cfg->model != RMHD_RESISTIVE && cfg->model != RMHD_TWO_FLUID) return RMHD_ERR_INVALID;
    if (cfg->nx < 1 || cfg->ny < 1 || (long long)cfg->nx * cfg->ny > (1LL << 31) - 1) return RMHD_ERR_INVALID;
    if (!(cfg->xmax > cfg->xmin) || (cfg->ny > 1 && !(cfg->ymax > cfg->ymin))) return RMHD_ERR_INVALID;
    if (!(cfg->gamma > 1.0 && cfg->gamma <= 2.0)) return RMHD_ERR_INVALID;
    if (!(cfg->sigma > 0.0) || !std::isfinite(cfg->sigma)) return RMHD_ERR_INVALID;
    if (!(cfg->kappa >= 0.0)) return RMHD_ERR_INVALID;
    if (cfg->model == RMHD_TWO_FLUID && !(cfg->mu_e != cfg->mu_p)) return RMHD_ERR_INVALID;
    if ((cfg->bc_x != RMHD_OUTFLOW && cfg->bc_x != RMHD_PERIODIC) || (cfg->bc_y != RMHD_OUTFLOW && cfg->bc_y != RMHD_PERIODIC))
        return RMHD_ERR_INVALID;
    if (cfg->precision != RMHD_FP64 && cfg->precision != RMHD_MIXED && cfg->precision != RMHD_FLOATFLOAT)
        return RMHD_ERR_INVALID;
    if (cfg->scheme != RMHD_SSP2 && cfg->scheme != RMHD_SSP3) return RMHD_ERR_INVALID;
    if (cfg->nz < 0) return RMHD_ERR_INVALID;
    // launch limits of the flux kernel's grid: tiles of 8 rows along y in
    // gridDim.y; in 3-D the z planes (x-y pass) and the y rows (z pass) in
    // gridDim.z, z in tiles of 8 rows in gridDim.y
    constexpr int kMaxGridYZ = 65535;
    if (cfg->ny > 1 && (cfg->ny + 7) / 8 > kMaxGridYZ) return RMHD_ERR_INVALID;
    if (cfg->nz > 1) {
        if (cfg->ny < 2 || !(cfg->zlen > 0.0)) return RMHD_ERR_INVALID;
        if (cfg->bc_z != RMHD_OUTFLOW && cfg->bc_z != RMHD_PERIODIC) return RMHD_ERR_INVALID;
        if ((long long)cfg->nx * cfg->ny * cfg->nz > (1LL << 31) - 1) return RMHD_ERR_INVALID;
        if (cfg->nz > kMaxGridYZ || cfg->ny > kMaxGridYZ) return RMHD_ERR_INVALID;
    }
    return RMHD_OK;
}

static Grid make_grid(const rmhd_config *cfg) {
    Grid g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.bcx = cfg->bc_x;
    g.bcy = cfg->bc_y;
    g.nz = cfg->nz > 1 ? cfg->nz : 1;
    g.bcz = cfg->bc_z;
    g.ncell = (long long)cfg->nx * cfg->ny * g.nz;
    g.plane = (g.ncell + 63) / 64 * 64;
    g.dx = (cfg->xmax - cfg->xmin) / cfg->nx;
    g.dy = cfg->ny > 1 ? (cfg->ymax - cfg->ymin) / cfg->ny : 1.0;
    g.dz = g.nz > 1 ? cfg->zlen / g.nz : 1.0;
    g.rdx4 = 0.25 / g.dx;
    g.rdy4 = 0.25 / g.dy;
    g.rdz4 = 0.25 / g.dz;
    g.row = cfg->nx;
    g.zoff = (long long)cfg->nx * cfg->ny;
    g.hlo = g.hhi = nullptr;
    return g;
}

struct Layout {
    size_t Q, W, Q1, W1, R, ACC, R3, LBUF, SRCG, stage, scratch, diag, status, hist, HLO, HHI, rlist;
    size_t nx, off, dx, rdx4, dt, sigma, eta, adt, cpsi, work, run_of, Qsave, Wsave;
    size_t total;
};

// Grid of a context; a batch is one packed 1-D "grid" of all runs' cells.
static Grid make_grid_n(const rmhd_config *cfg, long long ncell) {
    Grid g = {};
    g.nx = (int)ncell;
    g.ny = 1;
    g.bcx = cfg->bc_x;
    g.bcy = cfg->bc_y;
    g.ncell = ncell;
    g.plane = (ncell + 63) / 64 * 64;
    g.dx = 1.0;
    g.dy = 1.0;
    g.rdx4 = 0.25;
    g.rdy4 = 0.25;
    g.nz = 1;
    g.bcz = 0;
    g.dz = 1.0;
    g.rdz4 = 0.25;
    g.row = ncell;
    g.zoff = 0;
    return g;
}

static Layout layout_g(const rmhd_config *cfg, const Grid &g, int nruns, long long maxwork, bool halo = false);

// Cells of one stage whose first solve start may fail and be restarted in
// the restart kernel (more are reported as failed).
static int restart_capacity(long long ncell) { return (int)std::min<long long>(ncell, 1 << 18); }

static Layout layout(const rmhd_config *cfg, bool halo = false) { return layout_g(cfg, make_grid(cfg), 0, 0, halo); }

static Layout layout_g(const rmhd_config *cfg, const Grid &g, int nruns, long long maxwork, bool halo) {
    int nc = model_nc(cfg->model), nw = model_nw(cfg->model), np = model_np(cfg->model);
    size_t pl = (size_t)g.plane * sizeof(double);
    Layout L;
    size_t o = 0;
    L.Q = o; o += align256(nc * pl);
    L.W = o; o += align256(nw * pl);
    L.Q1 = o; o += align256(nc * pl);
    L.W1 = o; o += align256(nw * pl);
    L.R = o; o += align256(nc * pl);
    L.R3 = 0;
    if (cfg->scheme == RMHD_SSP3) { L.R3 = o; o += align256(nc * pl); }
    L.LBUF = 0;
    if (cfg->nz > 1) { L.LBUF = o; o += align256(nc * pl); }
    // planes the FP64 line-sweep pass takes from the stage kernel: one fluid J
    // (3), Z and p + (E^2 + B^2)/2; two fluids the source entries (7 used)
    L.SRCG = 0;
    if (nruns == 0) { L.SRCG = o; o += align256((cfg->model == RMHD_TWO_FLUID ? 9 : 5) * pl); }
    L.ACC = o; o += align256(nc * pl);
    L.stage = o; o += align256((size_t)std::max(nc, np) * g.ncell * sizeof(double));
    L.scratch = o; o += align256(reduce_scratch_doubles() * sizeof(double));
    L.diag = o; o += align256(8 * sizeof(double));
    L.status = o; o += align256(2 * sizeof(int));
    L.hist = o; o += align256(44 * sizeof(unsigned long long));
    L.rlist = o; o += align256((2 + (size_t)restart_capacity(g.ncell)) * sizeof(int));
    L.HLO = L.HHI = 0;
    if (halo) {  // slab: two halo rows of every staged variable below and above
        const size_t hb = (size_t)(nc + nw) * 2 * g.nx * sizeof(double);
        L.HLO = o; o += align256(hb);
        L.HHI = o; o += align256(hb);
    }
    L.nx = L.off = L.dx = L.rdx4 = L.dt = L.sigma = L.eta = L.adt = L.cpsi = L.work = L.run_of = L.Qsave = L.Wsave = 0;
    if (nruns > 0) {
        L.nx = o; o += align256((size_t)nruns * sizeof(int));
        L.off = o; o += align256((size_t)nruns * sizeof(long long));
        L.dx = o; o += align256((size_t)nruns * sizeof(double));
        L.rdx4 = o; o += align256((size_t)nruns * sizeof(double));
        L.dt = o; o += align256((size_t)nruns * sizeof(double));
        L.sigma = o; o += align256((size_t)nruns * sizeof(double));
        L.eta = o; o += align256((size_t)nruns * sizeof(double));
        L.adt = o; o += align256((size_t)nruns * sizeof(double));
        L.cpsi = o; o += align256((size_t)nruns * sizeof(double));
        L.work = o; o += align256((size_t)maxwork * sizeof(int2));
        L.run_of = o; o += align256((size_t)g.ncell * sizeof(int));
        L.Qsave = o; o += align256(nc * pl);
        L.Wsave = o; o += align256(nw * pl);
    }
    L.total = o;
    return L;
}

static long long batch_maxwork(int nruns, const int *nx) {
    long long w = 0;
    for (int r = 0; r < nruns; ++r) w += (nx[r] + 63) / 64;  // the narrowest tile width
    return w;
}

extern "C" {

const char *rmhd_version(void) { return "rmhd-gb300 0.1 (sm_103a)"; }

int rmhd_workspace_bytes(const rmhd_config *cfg, size_t *bytes) {
    if (!bytes) return RMHD_ERR_INVALID;
    int v = validate(cfg);
    if (v) return v;
    *bytes = layout(cfg).total;
    return RMHD_OK;
}

const char *rmhd_last_error(const rmhd_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

// Device status word: one 64-bit key (first failing cell << 8 | -code), all
// ones when no cell failed.
static int reset_status(rmhd_ctx *c) {
    CK(c, cudaMemsetAsync(c->status, 0xff, sizeof(unsigned long long), c->stream));
    return RMHD_OK;
}

// synchronise and decode the device status word
static int read_status(rmhd_ctx *c, const char *what) {
    CK(c, cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    unsigned long long key;
    memcpy(&key, c->h_status, sizeof key);
    if (key == ~0ull) return RMHD_OK;
    const int code = -(int)(key & 0xff);
    const long long cell = (long long)(key >> 8);
    int st = reset_status(c);
    if (st) return st;
    int i = (int)(cell % c->cfg.nx), j = (int)(cell / c->cfg.nx);
    const char *kind = code == RMHD_ERR_NEWTON ? "implicit-stage solve did not converge"
                       : code == RMHD_ERR_C2P  ? "primitive recovery failed"
                                               : "inadmissible primitive state";
    return fail(c, code, "%s: %s in cell (i=%d, j=%d)", what, kind, i, j);
}

static int create_impl(rmhd_ctx **out, const rmhd_config *cfg, void *cuda_stream, void *workspace,
                       size_t workspace_bytes, bool halo) {
    if (!out) return RMHD_ERR_INVALID;
    *out = nullptr;
    int v = validate(cfg);
    if (v) return v;
    rmhd_ctx *c = new rmhd_ctx();
    c->slab = false;
    c->slab_j0 = 0;
    c->slab_ny = cfg->ny;
    c->HLO = c->HHI = nullptr;
    c->phase_next = 0;
    c->phase_dt = 0.0;
    c->cfg = *cfg;
    c->g = make_grid(cfg);
    c->ph.gamma = cfg->gamma;
    c->ph.sigma = cfg->sigma;
    c->ph.kappa = cfg->kappa;
    c->ph.mu_e = cfg->mu_e;
    c->ph.mu_p = cfg->mu_p;
    c->ph.inv_dmu = cfg->model == RMHD_TWO_FLUID ? 1.0 / (cfg->mu_e - cfg->mu_p) : 0.0;
    c->ph.eta = 1.0 / cfg->sigma;
    c->ph.mur = std::max(std::fabs(cfg->mu_e), std::fabs(cfg->mu_p));
    if (!(c->ph.mur > 0.0)) c->ph.mur = 1.0;
    c->ph.imur = 1.0 / c->ph.mur;
    c->stream = (cudaStream_t)cuda_stream;
    c->graph = nullptr;
    c->graph_dt = 0.0;
    c->profiling = false;
    c->batch = false;
    c->nruns = 0;
    c->nwork = 0;
    c->h_tab = nullptr;
    c->tile_x = 128;
    c->flux_blocks = 0;
    c->stage_threads = 128;
    c->tab_dt = -1.0;
    c->recording = false;
    c->rec_ws = nullptr;
    c->rec_own = false;
    c->rec_nsteps = c->rec_K = c->rec_done = 0;
    c->rec_dt = 0.0;
    c->t = 0.0;
    c->has_state = false;
    c->fresh_prims = false;
    c->w_stale = false;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return RMHD_ERR_CUDA; }
    Layout L = layout(cfg, halo);
    if (workspace) {
        if (workspace_bytes < L.total || ((uintptr_t)workspace & 255)) { delete c; return RMHD_ERR_NOMEM; }
        c->ws = (char *)workspace;
        c->own_ws = false;
    } else {
        if (cudaMalloc(&c->ws, L.total) != cudaSuccess) { delete c; return RMHD_ERR_NOMEM; }
        c->own_ws = true;
    }
    c->ws_bytes = L.total;
    c->Q = (double *)(c->ws + L.Q);
    c->W = (double *)(c->ws + L.W);
    c->Q1 = (double *)(c->ws + L.Q1);
    c->W1 = (double *)(c->ws + L.W1);
    c->R = (double *)(c->ws + L.R);
    c->ACC = (double *)(c->ws + L.ACC);
    c->R3 = L.R3 ? (double *)(c->ws + L.R3) : nullptr;
    c->LBUF = L.LBUF ? (double *)(c->ws + L.LBUF) : nullptr;
    c->SRCG = L.SRCG ? (double *)(c->ws + L.SRCG) : nullptr;
    c->stage_buf = (double *)(c->ws + L.stage);
    c->scratch = (double *)(c->ws + L.scratch);
    c->diag = (double *)(c->ws + L.diag);
    c->status = (int *)(c->ws + L.status);
    c->hist = (unsigned long long *)(c->ws + L.hist);
    c->rlist = (int *)(c->ws + L.rlist);
    c->rcap = restart_capacity(c->g.ncell);
    if (halo) {
        c->HLO = (double *)(c->ws + L.HLO);
        c->HHI = (double *)(c->ws + L.HHI);
    }
    if (cudaMallocHost(&c->h_status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_diag, 8 * sizeof(double)) != cudaSuccess) {
        if (c->h_status) cudaFreeHost(c->h_status);  // the first may have succeeded
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return RMHD_ERR_NOMEM;
    }
    if (reset_status(c)) { rmhd_destroy(c); return RMHD_ERR_CUDA; }
    if (cudaMemsetAsync(c->rlist, 0, 2 * sizeof(int), c->stream) != cudaSuccess) {  // empty restart list
        rmhd_destroy(c);
        return RMHD_ERR_CUDA;
    }
    *out = c;
    return RMHD_OK;
}

int rmhd_create(rmhd_ctx **out, const rmhd_config *cfg, void *cuda_stream, void *workspace, size_t workspace_bytes) {
    return create_impl(out, cfg, cuda_stream, workspace, workspace_bytes, false);
}

// ---------------------------------------------------------------- slabs
// Configuration of the slab [j0, j0 + ny_local) of the global 2-D grid: the
// global x-range and cell widths, ny_local rows.
static int slab_config(const rmhd_config *global, int j0, int ny_local, rmhd_config *local) {
    int v = validate(global);
    if (v) return v;
    if (global->nz > 1 || global->ny < 2 || ny_local < 2 || j0 < 0 || j0 + ny_local > global->ny)
        return RMHD_ERR_INVALID;
    const double dy = (global->ymax - global->ymin) / global->ny;
    *local = *global;
    local->ny = ny_local;
    local->ymin = global->ymin + j0 * dy;
    local->ymax = global->ymin + (j0 + ny_local) * dy;
    return validate(local);
}

int rmhd_slab_workspace_bytes(const rmhd_config *global, int j0, int ny_local, size_t *bytes) {
    if (!bytes) return RMHD_ERR_INVALID;
    rmhd_config local;
    int v = slab_config(global, j0, ny_local, &local);
    if (v) return v;
    *bytes = layout(&local, true).total;
    return RMHD_OK;
}

int rmhd_create_slab(rmhd_ctx **out, const rmhd_config *global, int j0, int ny_local, void *cuda_stream,
                     void *workspace, size_t workspace_bytes) {
    if (!out) return RMHD_ERR_INVALID;
    *out = nullptr;
    rmhd_config local;
    int v = slab_config(global, j0, ny_local, &local);
    if (v) return v;
    rmhd_ctx *c = nullptr;
    v = create_impl(&c, &local, cuda_stream, workspace, workspace_bytes, true);
    if (v) return v;
    c->slab = true;
    c->slab_j0 = j0;
    c->slab_ny = global->ny;
    // the global cell height (the slab's own extent / ny_local may differ in the last bit)
    c->g.dy = (global->ymax - global->ymin) / global->ny;
    c->g.rdy4 = 0.25 / c->g.dy;
    // a side has a neighbour unless it is the global boundary with outflow
    const bool per = global->bc_y == RMHD_PERIODIC;
    c->g.hlo = (j0 > 0 || per) ? c->HLO : nullptr;
    c->g.hhi = (j0 + ny_local < global->ny || per) ? c->HHI : nullptr;
    c->g.bcy = RMHD_OUTFLOW;  // a side without a neighbour is a global outflow boundary
    c->cfg.bc_y = RMHD_OUTFLOW;
    *out = c;
    return RMHD_OK;
}

static bool has_halo(const rmhd_ctx *c) { return c->g.hlo || c->g.hhi; }

int rmhd_halo_doubles(const rmhd_ctx *c, size_t *n) {
    if (!c || !n) return RMHD_ERR_INVALID;
    if (!c->slab) return RMHD_ERR_STATE;
    *n = (size_t)(model_nc(c->cfg.model) + model_nw(c->cfg.model)) * 2 * c->g.nx;
    return RMHD_OK;
}

// The first two rows (lo) and the last two rows (hi) of the current stage
// state -- the state the next flux pass reads -- as [NC + NW][2][nx].
int rmhd_halo_pack(rmhd_ctx *c, double *lo, double *hi) {
    if (!c) return RMHD_ERR_INVALID;
    if (!c->slab) return fail(c, RMHD_ERR_STATE, "halo_pack: not a slab context");
    const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    const size_t w2 = 2 * (size_t)c->g.nx * sizeof(double), pl = (size_t)c->g.plane * sizeof(double);
    const size_t hi_off = (size_t)(c->g.ny - 2) * c->g.nx;
    const double *q = c->Q1, *w = c->W1;
    if (lo) {
        CK(c, cudaMemcpy2DAsync(lo, w2, q, pl, w2, nc, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemcpy2DAsync(lo + (size_t)nc * 2 * c->g.nx, w2, w, pl, w2, nw, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (hi) {
        CK(c, cudaMemcpy2DAsync(hi, w2, q + hi_off, pl, w2, nc, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemcpy2DAsync(hi + (size_t)nc * 2 * c->g.nx, w2, w + hi_off, pl, w2, nw, cudaMemcpyDeviceToDevice,
                                c->stream));
    }
    return RMHD_OK;
}

int rmhd_halo_unpack(rmhd_ctx *c, const double *lo, const double *hi) {
    if (!c) return RMHD_ERR_INVALID;
    if (!c->slab) return fail(c, RMHD_ERR_STATE, "halo_unpack: not a slab context");
    size_t n = 0;
    rmhd_halo_doubles(c, &n);
    if (lo && c->g.hlo) CK(c, cudaMemcpyAsync(c->HLO, lo, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (hi && c->g.hhi) CK(c, cudaMemcpyAsync(c->HHI, hi, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return RMHD_OK;
}

void rmhd_destroy(rmhd_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (auto &t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    if (c->own_ws) cudaFree(c->ws);
    cudaFreeHost(c->h_status);
    cudaFreeHost(c->h_diag);
    if (c->h_tab) cudaFreeHost(c->h_tab);
    if (c->rec_own && c->rec_ws) cudaFree(c->rec_ws);
    delete c;
}

// Bring user data [nvar][ny][nx] to the device staging buffer (dense layout).
static int stage_in(rmhd_ctx *c, const double *src, int nvar, int where) {
    size_t bytes = (size_t)nvar * c->g.ncell * sizeof(double);
    CK(c, cudaMemcpyAsync(c->stage_buf, src, bytes, where == RMHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          c->stream));
    return RMHD_OK;
}
static int stage_out(rmhd_ctx *c, double *dst, int nvar, int where) {
    size_t bytes = (size_t)nvar * c->g.ncell * sizeof(double);
    CK(c, cudaMemcpyAsync(dst, c->stage_buf, bytes, where == RMHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return RMHD_OK;
}

// Address at which this context's kernels can read or write a caller's buffer
// in place: a device buffer on the context's device as it is; page-locked
// host memory (cudaHostAlloc, cudaHostRegister, torch pinned tensors) through
// its mapping into the device's address space, so the kernels stream it over
// the host link with no staging copy. Null for pageable host memory, which
// goes through the staging buffer. A RMHD_DEVICE pointer that is not device
// memory of this device is an error (*bad set).
static void *device_view(const rmhd_ctx *c, const void *p, int where, bool *bad) {
    *bad = false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        *bad = where == RMHD_DEVICE;
        return nullptr;
    }
    if (where == RMHD_DEVICE) {
        if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != c->device) {
            *bad = true;
            return nullptr;
        }
        return const_cast<void *>(p);
    }
    // page-locked memory is mapped at its host address under unified
    // addressing; anything else is staged
    return a.type == cudaMemoryTypeHost && a.devicePointer == p ? a.devicePointer : nullptr;
}

// Device-readable view of a caller's input [nvar][cells]: the buffer itself
// where the device can address it, else the staging buffer after a copy.
static int input_view(rmhd_ctx *c, const double *src, int nvar, int where, const double **view, const char *what) {
    bool bad;
    if (void *d = device_view(c, src, where, &bad)) {
        *view = static_cast<const double *>(d);
        return RMHD_OK;
    }
    if (bad) return fail(c, RMHD_ERR_INVALID, "%s: RMHD_DEVICE pointer is not device memory of this context's device", what);
    int st = stage_in(c, src, nvar, where);
    *view = c->stage_buf;
    return st;
}

// Where an output kernel writes a caller's buffer: in place where the device
// can address it, else the staging buffer (finish_output copies it out).
static int output_view(rmhd_ctx *c, double *dst, int where, double **view, const char *what) {
    bool bad;
    void *d = device_view(c, dst, where, &bad);
    if (bad) return fail(c, RMHD_ERR_INVALID, "%s: RMHD_DEVICE pointer is not device memory of this context's device", what);
    *view = d ? static_cast<double *>(d) : c->stage_buf;
    return RMHD_OK;
}
// Completes an output written through output_view: the copy out of the
// staging buffer if one was used, then the stream is synchronised.
static int finish_output(rmhd_ctx *c, double *dst, const double *view, int nvar) {
    if (view == c->stage_buf)
        CK(c, cudaMemcpyAsync(dst, c->stage_buf, (size_t)nvar * c->g.ncell * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return RMHD_OK;
}

int rmhd_set_prims(rmhd_ctx *c, const double *prims, int where) {
    if (!c || !prims || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "set_prims: bad argument");
    if (has_halo(c))
        return fail(c, RMHD_ERR_STATE, "set_prims: Gauss's law at a slab's edge needs the neighbour's field; "
                                       "set a slab's state with rmhd_set_cons or rmhd_set_state");
    int np = model_np(c->cfg.model);
    const double *src;
    int st = input_view(c, prims, np, where, &src, "set_prims");
    if (st) return st;
    if (c->batch)
        CK(c, launch_set_prims_batch(c->cfg.model, c->g, c->ph, c->bargs, src, c->Q, c->W, c->status, c->stream));
    else
        CK(c, launch_set_prims(c->cfg.model, c->g, c->ph, src, c->Q, c->W, c->status, c->stream));
    st = read_status(c, "set_prims");
    if (st) return st;
    c->has_state = true;
    c->phase_next = 0;
    c->t = 0.0;
    c->recording = false;
    c->rec_done = 0;
    c->fresh_prims = true;
    c->w_stale = false;
    return RMHD_OK;
}

// A step leaves in W the stage-2 primitives (the next solve's warm start);
// the primitives of Q are recovered here when an output call needs them.
static int ensure_prims(rmhd_ctx *c, const char *what) {
    if (!c->w_stale) return RMHD_OK;
    CK(c, launch_recover(c->cfg.model, c->g, c->ph, c->Q, c->W, c->status, c->stream));
    int st = read_status(c, what);
    if (st) return st;
    c->w_stale = false;
    return RMHD_OK;
}

int rmhd_get_prims(rmhd_ctx *c, double *prims, int where) {
    if (!c || !prims || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "get_prims: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "get_prims: no state (call rmhd_set_prims first)");
    const int np = model_np(c->cfg.model);
    double *out;
    int st = output_view(c, prims, where, &out, "get_prims");
    if (st) return st;
    if (!c->w_stale) {
        CK(c, launch_get_prims(c->cfg.model, c->g, c->ph, c->Q, c->W, out, c->stream));
        return finish_output(c, prims, out, np);
    }
    // recovery and output in one kernel; the status is read after the copy
    CK(c, launch_recover(c->cfg.model, c->g, c->ph, c->Q, c->W, c->status, c->stream, out));
    if (out == c->stage_buf)
        CK(c, cudaMemcpyAsync(prims, c->stage_buf, (size_t)np * c->g.ncell * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    st = read_status(c, "get_prims");
    if (st) return st;
    c->w_stale = false;
    return RMHD_OK;
}

int rmhd_get_cons(rmhd_ctx *c, double *cons, int where) {
    if (!c || !cons || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "get_cons: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "get_cons: no state (call rmhd_set_prims first)");
    int nc = model_nc(c->cfg.model);
    double *out;
    int st = output_view(c, cons, where, &out, "get_cons");
    if (st) return st;
    CK(c, launch_unpack(c->g, nc, c->Q, out, c->stream));
    return finish_output(c, cons, out, nc);
}

int rmhd_set_cons(rmhd_ctx *c, const double *cons, int where) {
    if (!c || !cons || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "set_cons: bad argument");
    int nc = model_nc(c->cfg.model);
    const double *src;
    int st = input_view(c, cons, nc, where, &src, "set_cons");
    if (st) return st;
    CK(c, launch_pack(c->g, nc, src, c->Q, c->stream));
    CK(c, launch_recover(c->cfg.model, c->g, c->ph, c->Q, c->W, c->status, c->stream));
    st = read_status(c, "set_cons");
    if (st) return st;
    c->has_state = true;
    c->phase_next = 0;
    c->w_stale = false;
    return RMHD_OK;
}

int rmhd_state_doubles(const rmhd_ctx *c, size_t *n) {
    if (!c || !n) return RMHD_ERR_INVALID;
    *n = (size_t)(model_nc(c->cfg.model) + model_nw(c->cfg.model)) * (size_t)c->g.ncell;
    return RMHD_OK;
}

int rmhd_get_state(rmhd_ctx *c, double *state, int where) {
    if (!c || !state || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "get_state: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "get_state: no state (call rmhd_set_prims first)");
    const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    double *out;
    int st = output_view(c, state, where, &out, "get_state");
    if (st) return st;
    if (out != c->stage_buf) {  // both parts in place
        CK(c, launch_unpack(c->g, nc, c->Q, out, c->stream));
        CK(c, launch_unpack(c->g, nw, c->W, out + (size_t)nc * c->g.ncell, c->stream));
        return finish_output(c, state, out, nc + nw);
    }
    // the staging buffer holds one part at a time
    CK(c, launch_unpack(c->g, nc, c->Q, c->stage_buf, c->stream));
    st = finish_output(c, state, c->stage_buf, nc);
    if (st) return st;
    CK(c, launch_unpack(c->g, nw, c->W, c->stage_buf, c->stream));
    return finish_output(c, state + (size_t)nc * c->g.ncell, c->stage_buf, nw);
}

int rmhd_set_state(rmhd_ctx *c, const double *state, int where) {
    if (!c || !state || (where != RMHD_HOST && where != RMHD_DEVICE)) return fail(c, RMHD_ERR_INVALID, "set_state: bad argument");
    const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    const double *src;
    int st = input_view(c, state, nc, where, &src, "set_state");
    if (st) return st;
    CK(c, launch_pack(c->g, nc, src, c->Q, c->stream));
    // same stream: a staged second part overwrites the staging buffer after the pack above
    st = input_view(c, state + (size_t)nc * c->g.ncell, nw, where, &src, "set_state");
    if (st) return st;
    CK(c, launch_pack(c->g, nw, src, c->W, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->has_state = true;
    c->phase_next = 0;
    c->fresh_prims = false;
    c->w_stale = true;  // W is a warm start; output calls recover the primitives of Q
    c->recording = false;
    c->rec_done = 0;
    return RMHD_OK;
}

// Event bracket around one launch when profiling (no-op otherwise).
static int tic(rmhd_ctx *c, int kind) {
    if (!c->profiling) return RMHD_OK;
    rmhd_ctx::Timed t{kind, nullptr, nullptr};
    CK(c, cudaEventCreate(&t.a));
    CK(c, cudaEventCreate(&t.b));
    CK(c, cudaEventRecord(t.a, c->stream));
    c->timed.push_back(t);
    return RMHD_OK;
}
static int toc(rmhd_ctx *c) {
    if (!c->profiling) return RMHD_OK;
    CK(c, cudaEventRecord(c->timed.back().b, c->stream));
    return RMHD_OK;
}

#define LAUNCH(c, kind, call)           \
    do {                                \
        int st_ = tic((c), (kind));     \
        if (st_) return st_;            \
        CK((c), (call));                \
        st_ = toc(c);                   \
        if (st_) return st_;            \
    } while (0)

// Flux-pass arguments: the stage state (q, w), then outputs added one by one
// as out = base + dt (aL L + aS Psi).
// Coefficients carry the time step: dt > 0 for single grids; batches pass
// dt = 0 and get per-unit-dt coefficients, which the kernel scales by each
// run's own dt.
// Stage-solve arguments with the context's statistics and refinement settings.
static StageArgs stage_args(const rmhd_ctx *c, const double *r, const double *wwarm, double *q, double *w,
                            double adt) {
    // FP64, 2-D and 3-D grids: the stage kernel hands the stage state's current
    // (one fluid) or sources (two fluids) to the line-sweep flux pass
    const bool tf_src = c->cfg.precision == RMHD_FP64 && c->g.ny > 1;
    StageArgs a{r, wwarm, q, w, c->status, adt, c->stats_on ? c->hist : nullptr, c->maxpass,
                c->cfg.model == RMHD_RESISTIVE ? c->rlist : nullptr, c->rcap, c->first_start,
                tf_src ? c->SRCG : nullptr};
    return a;
}

static FluxArgs flux_args(const double *q, const double *w) {
    FluxArgs a{};
    a.q = q;
    a.w = w;
    return a;
}
static int add_out(FluxArgs &a, int k, const double *base, double *out, double aL, double aS, double dt) {
    const double sc = dt > 0.0 ? dt : 1.0;
    a.base[k] = base;
    a.out[k] = out;
    a.cL[k] = aL * sc;
    a.cS[k] = aS * sc;
    return k + 1;
}

// SSP2(222) flux passes (Table 1): pass 1 forms r2 = q^n + dt L1 + (1 - 2g) dt Psi1
// and acc = q^n + dt/2 (L1 + Psi1); pass 2 forms q^{n+1} = acc + dt/2 (L2 + Psi2).
static int ssp2_pass1(rmhd_ctx *c, const double *q1, const double *w1, double dt, FluxArgs &a) {
    a = flux_args(q1, w1);
    int n = add_out(a, 0, c->Q, c->R, 1.0, 1.0 - 2.0 * kGamma, dt);
    return add_out(a, n, c->Q, c->ACC, 0.5, 0.5, dt);
}
static int ssp2_pass2(rmhd_ctx *c, const double *q2, const double *w2, double dt, FluxArgs &a) {
    a = flux_args(q2, w2);
    a.wcarry = c->W;
    return add_out(a, 0, c->ACC, c->Q, 0.5, 0.5, dt);
}

// One SSP2(222) step of a batch: per-run dt, a_ii dt and 1/(1 + a_ii dt kappa)
// come from the device tables (uploaded by upload_dt_tables).
static int enqueue_step_batch(rmhd_ctx *c) {
    const int m = c->cfg.model;
    FluxArgs f;
    StageArgs s1 = stage_args(c, c->Q, c->W, c->Q1, c->W1, 0.0);
    LAUNCH(c, RMHD_K_STAGE, launch_stage_batch(m, c->g, c->ph, s1, c->bargs, c->stage_threads, c->stream));
    int n = ssp2_pass1(c, c->Q1, c->W1, 0.0, f);
    LAUNCH(c, RMHD_K_FLUX1, launch_flux_batch(m, c->cfg.precision, n, c->g, c->ph, f, c->bargs, c->tile_x,
                                              c->flux_blocks, c->stream));
    StageArgs s2 = stage_args(c, c->R, c->W1, c->Q1, c->W1, 0.0);
    LAUNCH(c, RMHD_K_STAGE, launch_stage_batch(m, c->g, c->ph, s2, c->bargs, c->stage_threads, c->stream));
    n = ssp2_pass2(c, c->Q1, c->W1, 0.0, f);
    LAUNCH(c, RMHD_K_FLUX2, launch_flux_batch(m, c->cfg.precision, n, c->g, c->ph, f, c->bargs, c->tile_x,
                                              c->flux_blocks, c->stream));
    return RMHD_OK;
}

// Per-run time-step tables: dt <= 0 selects each run's own CFL step.
static int upload_dt_tables(rmhd_ctx *c, double dt) {
    if (c->tab_dt == dt) return RMHD_OK;
    const int n = c->nruns;
    double *h = c->h_tab;
    for (int r = 0; r < n; ++r) {
        double d = dt > 0.0 ? dt : c->cfg.cfl * c->run_dx[r];
        h[r] = d;
        h[n + r] = kGamma * d;
        h[2 * n + r] = 1.0 / (1.0 + kGamma * d * c->cfg.kappa);
    }
    CK(c, cudaMemcpyAsync(c->d_dt, h, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_adt, h + n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->d_cpsi, h + 2 * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // the pinned staging must not be rewritten before these copies run
    CK(c, cudaStreamSynchronize(c->stream));
    c->tab_dt = dt;
    return RMHD_OK;
}

// One flux pass of a single grid (3-D grids take the two-pass path).
static cudaError_t flux_pass(rmhd_ctx *c, int nout, const FluxArgs &f0) {
    FluxArgs f = f0;
    f.srcg = c->SRCG;
    f.lscr = c->stage_buf;  // idle during steps (it serves the host I/O calls only)
    if (c->g.nz > 1) return launch_flux_3d(c->cfg.model, c->cfg.precision, nout, c->g, c->ph, f, c->LBUF, c->stream);
    return launch_flux(c->cfg.model, c->cfg.precision, nout, c->g, c->ph, f, c->stream);
}

// Smallest cell width (the CFL time step uses it).
static double min_width(const rmhd_ctx *c) {
    double h = c->g.dx;
    if (c->cfg.ny > 1) h = std::min(h, c->g.dy);
    if (c->g.nz > 1) h = std::min(h, c->g.dz);
    return h;
}

// Phases of one IMEX step: the implicit stage solves (even phases) and the
// flux passes (odd phases), in order. SSP2(222) (Table 1), 4 phases:
//   0: q1 = q^n + g dt Psi(q1)                       (stage solve into Q1/W1)
//   1: r2 = q^n + dt L1 + (1 - 2g) dt Psi1,  acc = q^n + dt/2 (L1 + Psi1)
//   2: q2 = r2 + g dt Psi(q2)                        (in place in Q1/W1)
//   3: q^{n+1} = acc + dt/2 (L2 + Psi2)              (stage-2 primitives kept as the warm start)
// SSP3(332) (Table 2), 6 phases: three stage solves (each in place in Q1/W1)
// and three flux passes:
//   pass 1: r2 = q^n + dt L1 + (1 - 2g) dt Psi1,  r3' = q^n + dt/4 L1 + (1/2 - g) dt Psi1,
//           acc = q^n + dt/6 (L1 + Psi1)
//   pass 2: r3 = r3' + dt/4 L2,  acc += dt/6 (L2 + Psi2)
//   pass 3: q^{n+1} = acc + 2 dt/3 (L3 + Psi3)
static int step_phases(const rmhd_ctx *c) { return c->cfg.scheme == RMHD_SSP3 ? 6 : 4; }

static int enqueue_phase(rmhd_ctx *c, double dt, int phase) {
    const int m = c->cfg.model;
    const bool ssp3 = c->cfg.scheme == RMHD_SSP3;
    const bool last = phase == step_phases(c) - 1;
    if ((phase & 1) == 0) {  // implicit stage solve: stage 1 from q^n, later stages from R
        StageArgs s = phase == 0 ? stage_args(c, c->Q, c->W, c->Q1, c->W1, kGamma * dt)
                                 : stage_args(c, c->R, c->W1, c->Q1, c->W1, kGamma * dt);
        LAUNCH(c, RMHD_K_STAGE, launch_stage(m, c->g, c->ph, s, c->stream));
        return RMHD_OK;
    }
    FluxArgs f;
    int n = 0;
    if (!ssp3) {
        n = phase == 1 ? ssp2_pass1(c, c->Q1, c->W1, dt, f) : ssp2_pass2(c, c->Q1, c->W1, dt, f);
    } else {
        f = flux_args(c->Q1, c->W1);
        if (phase == 1) {
            n = add_out(f, 0, c->Q, c->R, 1.0, 1.0 - 2.0 * kGamma, dt);
            n = add_out(f, n, c->Q, c->R3, 0.25, 0.5 - kGamma, dt);
            n = add_out(f, n, c->Q, c->ACC, 1.0 / 6.0, 1.0 / 6.0, dt);
        } else if (phase == 3) {
            n = add_out(f, 0, c->R3, c->R, 0.25, 0.0, dt);
            n = add_out(f, n, c->ACC, c->ACC, 1.0 / 6.0, 1.0 / 6.0, dt);
        } else {
            f.wcarry = c->W;
            n = add_out(f, 0, c->ACC, c->Q, 2.0 / 3.0, 2.0 / 3.0, dt);
        }
    }
    LAUNCH(c, last ? RMHD_K_FLUX2 : RMHD_K_FLUX1, flux_pass(c, n, f));
    return RMHD_OK;
}

// Enqueue one IMEX step with time step dt.
static int enqueue_step(rmhd_ctx *c, double dt) {
    if (c->batch) return enqueue_step_batch(c);
    for (int p = 0; p < step_phases(c); ++p) {
        int st = enqueue_phase(c, dt, p);
        if (st) return st;
    }
    return RMHD_OK;
}

int rmhd_step_phase(rmhd_ctx *c, double dt, int phase, double *t_out) {
    if (!c || phase < 0) return fail(c, RMHD_ERR_INVALID, "step_phase: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "step_phase: no state");
    if (c->batch || c->recording)
        return fail(c, RMHD_ERR_STATE, "step_phase: single grids without an armed recording only");
    if (phase >= step_phases(c)) return fail(c, RMHD_ERR_INVALID, "step_phase: phase %d of %d", phase, step_phases(c));
    if (phase != c->phase_next)
        return fail(c, RMHD_ERR_STATE, "step_phase: expected phase %d, got %d", c->phase_next, phase);
    if (phase == 0) {
        if (!(dt > 0.0)) dt = c->cfg.cfl * min_width(c);
        if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, RMHD_ERR_INVALID, "step_phase: dt must be positive");
        c->phase_dt = dt;
        c->fresh_prims = false;
    } else if (dt > 0.0 && dt != c->phase_dt) {
        return fail(c, RMHD_ERR_INVALID, "step_phase: the phases of a step take one dt (%g, got %g)", c->phase_dt, dt);
    }
    int st = enqueue_phase(c, c->phase_dt, phase);
    if (st) return st;
    c->phase_next = (phase + 1) % step_phases(c);
    if (c->phase_next == 0) {
        c->t += c->phase_dt;
        c->w_stale = true;
    }
    if (t_out) *t_out = c->t;
    return RMHD_OK;
}

int rmhd_imex_step(rmhd_ctx *c, double dt, int nsteps, double *t_out) {
    if (!c || nsteps < 0) return fail(c, RMHD_ERR_INVALID, "imex_step: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "imex_step: no state (call rmhd_set_prims first)");
    if (has_halo(c))
        return fail(c, RMHD_ERR_STATE, "imex_step: a slab with neighbours steps by rmhd_step_phase with halo exchange");
    if (c->phase_next != 0) return fail(c, RMHD_ERR_STATE, "imex_step: a phase-by-phase step is not finished");
    if (c->batch) {
        if (!(c->cfg.cfl > 0.0) && !(dt > 0.0)) return fail(c, RMHD_ERR_INVALID, "imex_step: dt <= 0 needs cfl > 0");
        int st = upload_dt_tables(c, dt > 0.0 ? dt : 0.0);
        if (st) return st;
        dt = dt > 0.0 ? dt : c->cfg.cfl * c->run_dx[0];  // time of run 0 is reported
    }
    if (!(dt > 0.0)) dt = c->cfg.cfl * min_width(c);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, RMHD_ERR_INVALID, "imex_step: dt must be positive (set cfl)");
    if (nsteps == 0) { if (t_out) *t_out = c->t; return RMHD_OK; }
    if (c->recording) {
        if (c->rec_done + nsteps > c->rec_nsteps)
            return fail(c, RMHD_ERR_STATE, "imex_step: more steps than the armed recording holds (%d)", c->rec_nsteps);
        if (c->rec_done > 0 && dt != c->rec_dt)
            return fail(c, RMHD_ERR_INVALID, "imex_step: a recorded run needs one dt (%g, got %g)", c->rec_dt, dt);
        c->rec_dt = dt;
        const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
        const size_t pl = (size_t)c->g.plane * sizeof(double);
        for (int n = 0; n < nsteps; ++n) {
            if (c->rec_done % c->rec_K == 0) {
                double *ck = c->rec_ck + (size_t)(c->rec_done / c->rec_K) * (nc + nw) * c->g.plane;
                CK(c, cudaMemcpyAsync(ck, c->Q, nc * pl, cudaMemcpyDeviceToDevice, c->stream));
                CK(c, cudaMemcpyAsync(ck + (size_t)nc * c->g.plane, c->W, nw * pl, cudaMemcpyDeviceToDevice, c->stream));
            }
            int st = enqueue_step(c, dt);
            if (st) return st;
            c->rec_done += 1;
            c->t += dt;
        }
        c->fresh_prims = false;
        c->w_stale = true;
        if (t_out) *t_out = c->t;
        return RMHD_OK;
    }
    c->fresh_prims = false;
    c->w_stale = true;
    // Legacy default stream (no graph capture there) or profiling: launch directly.
    if (c->profiling || c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread) {
        for (int n = 0; n < nsteps; ++n) {
            int st = enqueue_step(c, dt);
            if (st) return st;
            c->t += dt;
        }
        if (t_out) *t_out = c->t;
        return RMHD_OK;
    }
    // one step as a CUDA graph, re-captured when dt changes
    if (!c->graph || c->graph_dt != dt) {
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
        // first launch outside capture also sets the kernels' shared-memory attributes
        int st = enqueue_step(c, dt);
        if (st) return st;
        nsteps -= 1;
        c->t += dt;
        cudaGraph_t gr;
        CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_step(c, dt);
        cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
        if (st) {
            if (e == cudaSuccess) cudaGraphDestroy(gr);
            return st;
        }
        if (e != cudaSuccess) return fail(c, RMHD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) { c->graph = nullptr; return fail(c, RMHD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        c->graph_dt = dt;
    }
    for (int n = 0; n < nsteps; ++n) {
        CK(c, cudaGraphLaunch(c->graph, c->stream));
        c->t += dt;
    }
    if (t_out) *t_out = c->t;
    return RMHD_OK;
}

// ---------------------------------------------------------------- batched ensemble
static int validate_batch(const rmhd_config *base, int nruns, const int *nx, const double *sigma) {
    if (!base || nruns < 1 || !nx) return RMHD_ERR_INVALID;
    rmhd_config one = *base;
    one.ny = 1;
    long long tot = 0;
    for (int r = 0; r < nruns; ++r) {
        if (nx[r] < 1) return RMHD_ERR_INVALID;
        tot += nx[r];
        if (sigma && !(sigma[r] > 0.0 && std::isfinite(sigma[r]))) return RMHD_ERR_INVALID;
    }
    if (tot > (1LL << 31) - 1) return RMHD_ERR_INVALID;
    if (base->scheme != RMHD_SSP2 || base->nz > 1) return RMHD_ERR_INVALID;
    if (base->precision == RMHD_FLOATFLOAT) return RMHD_ERR_INVALID;  // batches: FP64 or mixed
    one.nx = (int)std::min<long long>(tot, 1 << 30);
    return validate(&one);
}

static long long batch_cells(int nruns, const int *nx) {
    long long t = 0;
    for (int r = 0; r < nruns; ++r) t += nx[r];
    return t;
}

int rmhd_batch_workspace_bytes(const rmhd_config *base, int nruns, const int *nx, size_t *bytes) {
    if (!bytes) return RMHD_ERR_INVALID;
    int v = validate_batch(base, nruns, nx, nullptr);
    if (v) return v;
    Grid g = make_grid_n(base, batch_cells(nruns, nx));
    *bytes = layout_g(base, g, nruns, batch_maxwork(nruns, nx)).total;
    return RMHD_OK;
}

// Work list of (run, first cell) tiles of width tile_x.
static int upload_work(rmhd_ctx *c, int tile_x) {
    std::vector<int2> w;
    for (int r = 0; r < c->nruns; ++r)
        for (int i0 = 0; i0 < c->run_nx[r]; i0 += tile_x) w.push_back(make_int2(r, i0));
    CK(c, cudaMemcpy(c->d_work, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice));
    c->nwork = (int)w.size();
    c->bargs.nwork = c->nwork;
    c->tile_x = tile_x;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return RMHD_OK;
}

static int default_blocks(rmhd_ctx *c, int tile_x) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    int occ = flux_batch_occupancy(c->cfg.model, c->cfg.precision, tile_x);
    return std::max(1, sms * std::max(1, occ));
}

int rmhd_create_batch(rmhd_ctx **out, const rmhd_config *base, int nruns, const int *nx, const double *sigma,
                      void *cuda_stream, void *workspace, size_t workspace_bytes) {
    if (!out) return RMHD_ERR_INVALID;
    *out = nullptr;
    int v = validate_batch(base, nruns, nx, sigma);
    if (v) return v;
    rmhd_config cfg = *base;
    cfg.ny = 1;
    cfg.nx = 1;  // placeholder; the packed grid is built below
    rmhd_ctx *c = nullptr;
    // create a single-run context for the bookkeeping, then re-lay it out as a batch
    Grid g = make_grid_n(&cfg, batch_cells(nruns, nx));
    Layout L = layout_g(&cfg, g, nruns, batch_maxwork(nruns, nx));
    if (workspace && workspace_bytes < L.total) return RMHD_ERR_NOMEM;
    cfg.nx = 1;
    int st = rmhd_create(&c, &cfg, cuda_stream, nullptr, 0);
    if (st) return st;
    // replace the single-run workspace with the batch one
    if (c->own_ws) cudaFree(c->ws);
    if (workspace) {
        if ((uintptr_t)workspace & 255) { c->own_ws = false; rmhd_destroy(c); return RMHD_ERR_NOMEM; }
        c->ws = (char *)workspace;
        c->own_ws = false;
    } else {
        if (cudaMalloc(&c->ws, L.total) != cudaSuccess) { c->own_ws = false; rmhd_destroy(c); return RMHD_ERR_NOMEM; }
        c->own_ws = true;
    }
    c->ws_bytes = L.total;
    c->g = g;
    c->cfg.nx = (int)g.ncell;  // messages name the packed cell index
    c->batch = true;
    c->nruns = nruns;
    c->Q = (double *)(c->ws + L.Q);
    c->W = (double *)(c->ws + L.W);
    c->Q1 = (double *)(c->ws + L.Q1);
    c->W1 = (double *)(c->ws + L.W1);
    c->R = (double *)(c->ws + L.R);
    c->ACC = (double *)(c->ws + L.ACC);
    c->R3 = L.R3 ? (double *)(c->ws + L.R3) : nullptr;
    c->LBUF = L.LBUF ? (double *)(c->ws + L.LBUF) : nullptr;
    c->SRCG = L.SRCG ? (double *)(c->ws + L.SRCG) : nullptr;
    c->stage_buf = (double *)(c->ws + L.stage);
    c->scratch = (double *)(c->ws + L.scratch);
    c->diag = (double *)(c->ws + L.diag);
    c->status = (int *)(c->ws + L.status);
    c->hist = (unsigned long long *)(c->ws + L.hist);
    c->rlist = (int *)(c->ws + L.rlist);
    c->rcap = restart_capacity(c->g.ncell);
    if (cudaMemsetAsync(c->rlist, 0, 2 * sizeof(int), c->stream) != cudaSuccess) {  // empty restart list
        rmhd_destroy(c);
        return RMHD_ERR_CUDA;
    }
    c->d_nx = (int *)(c->ws + L.nx);
    c->d_off = (long long *)(c->ws + L.off);
    c->d_dx = (double *)(c->ws + L.dx);
    c->d_rdx4 = (double *)(c->ws + L.rdx4);
    c->d_dt = (double *)(c->ws + L.dt);
    c->d_sigma = (double *)(c->ws + L.sigma);
    c->d_eta = (double *)(c->ws + L.eta);
    c->d_adt = (double *)(c->ws + L.adt);
    c->d_cpsi = (double *)(c->ws + L.cpsi);
    c->d_work = (int2 *)(c->ws + L.work);
    c->d_run_of = (int *)(c->ws + L.run_of);
    c->Qsave = (double *)(c->ws + L.Qsave);
    c->Wsave = (double *)(c->ws + L.Wsave);
    c->run_nx.assign(nx, nx + nruns);
    c->run_off.resize(nruns);
    c->run_dx.resize(nruns);
    c->run_sigma.resize(nruns);
    std::vector<int> run_of(g.ncell);
    std::vector<double> eta(nruns), rdx4(nruns);
    long long o = 0;
    for (int r = 0; r < nruns; ++r) {
        c->run_off[r] = o;
        c->run_dx[r] = (base->xmax - base->xmin) / nx[r];
        c->run_sigma[r] = sigma ? sigma[r] : base->sigma;
        eta[r] = 1.0 / c->run_sigma[r];
        rdx4[r] = 0.25 / c->run_dx[r];
        for (int i = 0; i < nx[r]; ++i) run_of[o + i] = r;
        o += nx[r];
    }
    if (cudaMallocHost(&c->h_tab, 3 * (size_t)nruns * sizeof(double)) != cudaSuccess) { rmhd_destroy(c); return RMHD_ERR_NOMEM; }
    bool ok = cudaMemcpy(c->d_nx, nx, nruns * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_off, c->run_off.data(), nruns * sizeof(long long), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_dx, c->run_dx.data(), nruns * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_rdx4, rdx4.data(), nruns * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_sigma, c->run_sigma.data(), nruns * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_eta, eta.data(), nruns * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->d_run_of, run_of.data(), g.ncell * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok || reset_status(c)) { rmhd_destroy(c); return RMHD_ERR_CUDA; }
    BatchArgs &b = c->bargs;
    b.nruns = nruns;
    b.work = c->d_work;
    b.nx = c->d_nx;
    b.offset = c->d_off;
    b.dx = c->d_dx;
    b.rdx4 = c->d_rdx4;
    b.dt = c->d_dt;
    b.sigma = c->d_sigma;
    b.eta = c->d_eta;
    b.adt = c->d_adt;
    b.cpsi = c->d_cpsi;
    b.run_of = c->d_run_of;
    if (upload_work(c, 128)) { rmhd_destroy(c); return RMHD_ERR_CUDA; }
    c->flux_blocks = default_blocks(c, 128);
    *out = c;
    return RMHD_OK;
}

// Time `reps` steps of the current configuration (state restored by the caller).
static int time_steps(rmhd_ctx *c, int reps, float *ms) {
    cudaEvent_t a, b;
    CK(c, cudaEventCreate(&a));
    CK(c, cudaEventCreate(&b));
    int st = enqueue_step(c, 0.0);  // warm-up (and per-kernel attribute set-up)
    if (!st) {
        cudaEventRecord(a, c->stream);
        for (int k = 0; k < reps && !st; ++k) st = enqueue_step(c, 0.0);
        cudaEventRecord(b, c->stream);
        if (!st) st = cudaEventSynchronize(b) == cudaSuccess ? RMHD_OK : RMHD_ERR_CUDA;
        if (!st) cudaEventElapsedTime(ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

int rmhd_autotune(rmhd_ctx *c, int *choice) {
    if (!c || !choice) return fail(c, RMHD_ERR_INVALID, "autotune: bad argument");
    if (!c->batch) return fail(c, RMHD_ERR_STATE, "autotune: only batched contexts are tuned");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "autotune: no state (call rmhd_set_prims first)");
    int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    size_t qb = (size_t)nc * c->g.plane * sizeof(double), wb = (size_t)nw * c->g.plane * sizeof(double);
    CK(c, cudaMemcpyAsync(c->Qsave, c->Q, qb, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->Wsave, c->W, wb, cudaMemcpyDeviceToDevice, c->stream));
    int st = upload_dt_tables(c, c->tab_dt > 0.0 ? c->tab_dt : 0.0);
    if (st) return st;
    bool prof = c->profiling;
    c->profiling = false;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    float best = 1e30f;
    int bt = 128, bb = default_blocks(c, 128), bs = 128;
    const int tiles[3] = {64, 128, 256};
    for (int ti = 0; ti < 3 && !st; ++ti) {
        int occ = flux_batch_occupancy(c->cfg.model, c->cfg.precision, tiles[ti]);
        if (occ < 1) continue;
        st = upload_work(c, tiles[ti]);
        for (int k = 1; k <= occ && !st; k *= 2) {
            c->flux_blocks = sms * k;
            float ms = 0.f;
            st = time_steps(c, 2, &ms);
            if (!st && ms < best) { best = ms; bt = tiles[ti]; bb = c->flux_blocks; }
            CK(c, cudaMemcpyAsync(c->Q, c->Qsave, qb, cudaMemcpyDeviceToDevice, c->stream));
            CK(c, cudaMemcpyAsync(c->W, c->Wsave, wb, cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    if (!st) st = upload_work(c, bt);
    c->flux_blocks = bb;
    const int threads[3] = {64, 128, 256};
    best = 1e30f;
    for (int k = 0; k < 3 && !st; ++k) {
        c->stage_threads = threads[k];
        float ms = 0.f;
        st = time_steps(c, 2, &ms);
        if (!st && ms < best) { best = ms; bs = threads[k]; }
        CK(c, cudaMemcpyAsync(c->Q, c->Qsave, qb, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->W, c->Wsave, wb, cudaMemcpyDeviceToDevice, c->stream));
    }
    c->stage_threads = bs;
    c->profiling = prof;
    CK(c, cudaStreamSynchronize(c->stream));
    if (st) return st;
    // the timing steps may have recorded failures of their own; the restored state is what counts
    st = reset_status(c);
    if (st) return st;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    choice[0] = c->tile_x;
    choice[1] = c->flux_blocks;
    choice[2] = c->stage_threads;
    return RMHD_OK;
}

// ---------------------------------------------------------------- discrete adjoint
struct RecLayout {
    size_t ck, seg, lam, lamn, lq, lr2, lr3, fx, fy, fz, fbx, fby, fbz, qbd, sig, pbar, fin, sum, total;
};

// implicit stages per step of the context's scheme
static int scheme_stages(const rmhd_ctx *c) { return c->cfg.scheme == RMHD_SSP3 ? 3 : 2; }

static RecLayout rec_layout(const rmhd_ctx *c, int nsteps, int K) {
    const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    const size_t pl = (size_t)c->g.plane * sizeof(double);
    const int nck = (nsteps + K - 1) / K;
    RecLayout L;
    size_t o = 0;
    L.ck = o; o += align256((size_t)nck * (nc + nw) * pl);
    L.seg = o; o += align256((size_t)K * scheme_stages(c) * (nc + nw) * pl);
    L.lam = o; o += align256(nc * pl);
    L.lamn = o; o += align256(nc * pl);
    L.lq = o; o += align256(nc * pl);
    L.lr2 = o; o += align256(nc * pl);
    L.lr3 = o; o += align256(nc * pl);
    const size_t zpl = c->g.nz > 1 ? nc * pl : 0;  // z fluxes: 3-D grids only
    L.fx = o; o += align256(nc * pl);
    L.fy = o; o += align256(nc * pl);
    L.fz = o; o += align256(zpl);
    L.fbx = o; o += align256(nc * pl);
    L.fby = o; o += align256(nc * pl);
    L.fbz = o; o += align256(zpl);
    L.qbd = o; o += align256(nc * pl);
    L.sig = o; o += align256(pl);
    L.pbar = o; o += align256(model_np(c->cfg.model) * pl);
    L.fin = o; o += align256((size_t)(nc + nw) * pl);
    L.sum = o; o += align256(sizeof(double));
    L.total = o;
    return L;
}

static int adjoint_supported(rmhd_ctx *c) {
    if (c->cfg.precision != RMHD_FP64 || c->batch || c->slab)
        return fail(c, RMHD_ERR_STATE, "adjoint: FP64 single-grid contexts only");
    if (c->cfg.nx < 3 || (c->cfg.ny > 1 && c->cfg.ny < 3) || (c->g.nz > 1 && c->g.nz < 3))
        return fail(c, RMHD_ERR_INVALID, "adjoint: grids need at least 3 cells per direction");
    return RMHD_OK;
}

int rmhd_recording_bytes(rmhd_ctx *c, int nsteps, int ckpt_every, size_t *bytes) {
    if (!c || !bytes || nsteps < 1 || ckpt_every < 1) return fail(c, RMHD_ERR_INVALID, "recording_bytes: bad argument");
    int st = adjoint_supported(c);
    if (st) return st;
    *bytes = rec_layout(c, nsteps, ckpt_every).total;
    return RMHD_OK;
}

int rmhd_record(rmhd_ctx *c, int nsteps, int ckpt_every, void *workspace, size_t bytes) {
    if (!c || nsteps < 1 || ckpt_every < 1) return fail(c, RMHD_ERR_INVALID, "record: bad argument");
    int st = adjoint_supported(c);
    if (st) return st;
    if (!c->has_state || !c->fresh_prims)
        return fail(c, RMHD_ERR_STATE, "record: arm right after rmhd_set_prims (the gradient is w.r.t. those primitives)");
    RecLayout L = rec_layout(c, nsteps, ckpt_every);
    // disarm any earlier recording first: a failure below must not leave the
    // context recording into a workspace that is gone
    c->recording = false;
    c->rec_done = 0;
    if (c->rec_own && c->rec_ws) { cudaFree(c->rec_ws); c->rec_ws = nullptr; c->rec_own = false; }
    if (workspace) {
        if (bytes < L.total || ((uintptr_t)workspace & 255)) return fail(c, RMHD_ERR_NOMEM, "record: workspace too small");
        c->rec_ws = (char *)workspace;
        c->rec_own = false;
    } else {
        if (cudaMalloc(&c->rec_ws, L.total) != cudaSuccess) return fail(c, RMHD_ERR_NOMEM, "record: allocation failed");
        c->rec_own = true;
    }
    c->rec_ck = (double *)(c->rec_ws + L.ck);
    c->rec_seg = (double *)(c->rec_ws + L.seg);
    c->rec_lam = (double *)(c->rec_ws + L.lam);
    c->rec_lamn = (double *)(c->rec_ws + L.lamn);
    c->rec_lq = (double *)(c->rec_ws + L.lq);
    c->rec_lr2 = (double *)(c->rec_ws + L.lr2);
    c->rec_lr3 = (double *)(c->rec_ws + L.lr3);
    c->rec_fx = (double *)(c->rec_ws + L.fx);
    c->rec_fy = (double *)(c->rec_ws + L.fy);
    c->rec_fz = (double *)(c->rec_ws + L.fz);
    c->rec_fbx = (double *)(c->rec_ws + L.fbx);
    c->rec_fby = (double *)(c->rec_ws + L.fby);
    c->rec_fbz = (double *)(c->rec_ws + L.fbz);
    c->rec_qbd = (double *)(c->rec_ws + L.qbd);
    c->rec_sig = (double *)(c->rec_ws + L.sig);
    c->rec_pbar = (double *)(c->rec_ws + L.pbar);
    c->rec_fin = (double *)(c->rec_ws + L.fin);
    c->rec_sum = (double *)(c->rec_ws + L.sum);
    c->recording = true;
    c->rec_nsteps = nsteps;
    c->rec_K = ckpt_every;
    c->rec_done = 0;
    c->rec_dt = 0.0;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return RMHD_OK;
}

// One forward step writing the stage states into caller buffers (same kernels
// and arithmetic as enqueue_step, so the recomputation reproduces the run):
// stage i into (Sq[i], Sw[i]).
static int enqueue_step_into(rmhd_ctx *c, double dt, double *const *Sq, double *const *Sw) {
    const int m = c->cfg.model;
    FluxArgs f;
    if (c->cfg.scheme == RMHD_SSP3) {
        // as enqueue_step_ssp3; stage 2 starts from stage 1's primitives, stage 3 from stage 2's
        StageArgs s1 = stage_args(c, c->Q, c->W, Sq[0], Sw[0], kGamma * dt);
        CK(c, launch_stage(m, c->g, c->ph, s1, c->stream));
        f = flux_args(Sq[0], Sw[0]);
        int n = add_out(f, 0, c->Q, c->R, 1.0, 1.0 - 2.0 * kGamma, dt);
        n = add_out(f, n, c->Q, c->R3, 0.25, 0.5 - kGamma, dt);
        n = add_out(f, n, c->Q, c->ACC, 1.0 / 6.0, 1.0 / 6.0, dt);
        CK(c, flux_pass(c, n, f));
        StageArgs s2 = stage_args(c, c->R, Sw[0], Sq[1], Sw[1], kGamma * dt);
        CK(c, launch_stage(m, c->g, c->ph, s2, c->stream));
        f = flux_args(Sq[1], Sw[1]);
        n = add_out(f, 0, c->R3, c->R, 0.25, 0.0, dt);
        n = add_out(f, n, c->ACC, c->ACC, 1.0 / 6.0, 1.0 / 6.0, dt);
        CK(c, flux_pass(c, n, f));
        StageArgs s3 = stage_args(c, c->R, Sw[1], Sq[2], Sw[2], kGamma * dt);
        CK(c, launch_stage(m, c->g, c->ph, s3, c->stream));
        f = flux_args(Sq[2], Sw[2]);
        f.wcarry = c->W;
        n = add_out(f, 0, c->ACC, c->Q, 2.0 / 3.0, 2.0 / 3.0, dt);
        CK(c, flux_pass(c, n, f));
        return RMHD_OK;
    }
    StageArgs s1 = stage_args(c, c->Q, c->W, Sq[0], Sw[0], kGamma * dt);
    CK(c, launch_stage(m, c->g, c->ph, s1, c->stream));
    int n = ssp2_pass1(c, Sq[0], Sw[0], dt, f);
    CK(c, flux_pass(c, n, f));
    StageArgs s2 = stage_args(c, c->R, Sw[0], Sq[1], Sw[1], kGamma * dt);
    CK(c, launch_stage(m, c->g, c->ph, s2, c->stream));
    n = ssp2_pass2(c, Sq[1], Sw[1], dt, f);
    CK(c, flux_pass(c, n, f));
    return RMHD_OK;
}

int rmhd_adjoint_step(rmhd_ctx *c, const double *dJ_dcons, int where_in, double *dJ_dprims0, int where_out,
                      double *dJ_dsigma) {
    if (!c || !dJ_dcons || (where_in != RMHD_HOST && where_in != RMHD_DEVICE) ||
        (dJ_dprims0 && where_out != RMHD_HOST && where_out != RMHD_DEVICE))
        return fail(c, RMHD_ERR_INVALID, "adjoint_step: bad argument");
    int st = adjoint_supported(c);
    if (st) return st;
    if (!c->recording || c->rec_done < 1) return fail(c, RMHD_ERR_STATE, "adjoint_step: no recorded steps (rmhd_record)");
    const int nc = model_nc(c->cfg.model), nw = model_nw(c->cfg.model);
    const size_t pl = (size_t)c->g.plane * sizeof(double);
    const long long P = c->g.plane;
    const double dt = c->rec_dt;
    // lambda^N = dJ/dq^N
    st = stage_in(c, dJ_dcons, nc, where_in);
    if (st) return st;
    CK(c, launch_pack(c->g, nc, c->stage_buf, c->rec_lam, c->stream));
    // keep the final state
    CK(c, cudaMemcpyAsync(c->rec_fin, c->Q, nc * pl, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->rec_fin + (size_t)nc * P, c->W, nw * pl, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->rec_sig, 0, pl, c->stream));
    const int K = c->rec_K, nseg = (c->rec_done + K - 1) / K;
    double *lam = c->rec_lam, *lamn = c->rec_lamn;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * K, len = std::min(K, c->rec_done - s0);
        const double *ck = c->rec_ck + (size_t)seg * (nc + nw) * P;
        CK(c, cudaMemcpyAsync(c->Q, ck, nc * pl, cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaMemcpyAsync(c->W, ck + (size_t)nc * P, nw * pl, cudaMemcpyDeviceToDevice, c->stream));
        const int S = scheme_stages(c);
        // stage i of step s: q at b + i (nc + nw) P, w right after it
        auto stage_ptrs = [&](int s, double **Sq, double **Sw) {
            double *b = c->rec_seg + (size_t)s * S * (nc + nw) * P;
            for (int k = 0; k < S; ++k) {
                Sq[k] = b + (size_t)k * (nc + nw) * P;
                Sw[k] = Sq[k] + (size_t)nc * P;
            }
        };
        for (int s = 0; s < len; ++s) {
            double *Sq[3], *Sw[3];
            stage_ptrs(s, Sq, Sw);
            st = enqueue_step_into(c, dt, Sq, Sw);
            if (st) return st;
        }
        for (int s = len - 1; s >= 0; --s) {
            double *Sq[3], *Sw[3];
            stage_ptrs(s, Sq, Sw);
            const double *cq[3] = {Sq[0], Sq[1], S > 2 ? Sq[2] : nullptr};
            const double *cw[3] = {Sw[0], Sw[1], S > 2 ? Sw[2] : nullptr};
            double *fl[3] = {c->rec_fx, c->rec_fy, c->rec_fz}, *fbl[3] = {c->rec_fbx, c->rec_fby, c->rec_fbz};
            CK(c, launch_adjoint_step(c->cfg.model, c->g, c->ph, S > 2 ? 1 : 0, dt, lam, lamn, cq, cw, fl, fbl, c->rec_qbd,
                                      c->rec_lq, c->rec_lr2, c->rec_lr3, c->rec_sig, c->stream));
            std::swap(lam, lamn);
        }
    }
    // initial primitives: adjoint of the prims -> cons map at checkpoint 0
    CK(c, launch_adjoint_prims(c->cfg.model, c->g, c->ph, c->rec_ck, c->rec_ck + (size_t)nc * P, lam, c->rec_pbar, c->stream));
    CK(c, launch_sum(c->rec_sig, c->g.ncell, c->rec_sum, c->stream));
    if (dJ_dprims0) {
        const int np = model_np(c->cfg.model);
        CK(c, launch_unpack(c->g, np, c->rec_pbar, c->stage_buf, c->stream));
        st = stage_out(c, dJ_dprims0, np, where_out);
        if (st) return st;
    }
    CK(c, cudaMemcpyAsync(c->h_diag, c->rec_sum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(c->Q, c->rec_fin, nc * pl, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->W, c->rec_fin + (size_t)nc * P, nw * pl, cudaMemcpyDeviceToDevice, c->stream));
    st = read_status(c, "adjoint_step");
    if (st) return st;
    if (dJ_dsigma) *dJ_dsigma = c->h_diag[0];
    return RMHD_OK;
}

int rmhd_set_profiling(rmhd_ctx *c, int enable) {
    if (!c) return RMHD_ERR_INVALID;
    c->profiling = enable != 0;
    return RMHD_OK;
}

int rmhd_kernel_times(rmhd_ctx *c, double *ms, int *counts) {
    if (!c || !ms || !counts) return fail(c, RMHD_ERR_INVALID, "kernel_times: bad argument");
    CK(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) { ms[k] = 0.0; counts[k] = 0; }
    int st = RMHD_OK;
    for (auto &t : c->timed) {
        float e = 0.f;
        if (st == RMHD_OK && cudaEventElapsedTime(&e, t.a, t.b) != cudaSuccess)
            st = fail(c, RMHD_ERR_CUDA, "kernel_times: cudaEventElapsedTime failed");
        ms[t.kind] += e;
        counts[t.kind] += 1;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->timed.clear();
    return st;
}

int rmhd_set_solver_stats(rmhd_ctx *c, int enable) {
    if (!c) return RMHD_ERR_INVALID;
    if (enable) CK(c, cudaMemsetAsync(c->hist, 0, 44 * sizeof(unsigned long long), c->stream));
    c->stats_on = enable != 0;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }  // captured with the old arguments
    CK(c, cudaStreamSynchronize(c->stream));
    return RMHD_OK;
}

int rmhd_solver_stats(rmhd_ctx *c, unsigned long long *hist) {
    if (!c || !hist) return fail(c, RMHD_ERR_INVALID, "solver_stats: bad argument");
    CK(c, cudaMemcpyAsync(hist, c->hist, 44 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemsetAsync(c->hist, 0, 44 * sizeof(unsigned long long), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return RMHD_OK;
}

int rmhd_set_refinement_cap(rmhd_ctx *c, int passes) {
    if (!c) return RMHD_ERR_INVALID;
    if (passes < 0 || passes > 8) return fail(c, RMHD_ERR_INVALID, "set_refinement_cap: passes must be 0..8");
    c->maxpass = passes;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }  // captured with the old arguments
    return RMHD_OK;
}

int rmhd_set_first_start(rmhd_ctx *c, int start) {
    if (!c || start < 0 || start > 2) return fail(c, RMHD_ERR_INVALID, "set_first_start: start must be 0, 1 or 2");
    if (c->cfg.model != RMHD_RESISTIVE) return fail(c, RMHD_ERR_STATE, "set_first_start: single-fluid contexts only");
    const long long cells = c->g.ncell;
    if (start > 0 && cells > c->rcap)
        return fail(c, RMHD_ERR_INVALID, "set_first_start: more cells (%lld) than the restart list holds (%d)", cells,
                    c->rcap);
    c->first_start = start;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }  // captured with the old arguments
    return RMHD_OK;
}

int rmhd_check(rmhd_ctx *c) {
    if (!c) return RMHD_ERR_INVALID;
    return read_status(c, "imex_step");
}

int rmhd_diagnostics(rmhd_ctx *c, double *out) {
    if (!c || !out) return fail(c, RMHD_ERR_INVALID, "diagnostics: bad argument");
    if (!c->has_state) return fail(c, RMHD_ERR_STATE, "diagnostics: no state");
    int st = ensure_prims(c, "diagnostics");
    if (st) return st;
    CK(c, launch_diagnostics(c->cfg.model, c->g, c->ph, c->Q, c->W, c->scratch, c->diag, c->stream));
    CK(c, cudaMemcpyAsync(c->h_diag, c->diag, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 7; ++k) out[k] = c->h_diag[k];
    out[7] = c->cfg.cfl * min_width(c);
    return RMHD_OK;
}

} // extern "C"
