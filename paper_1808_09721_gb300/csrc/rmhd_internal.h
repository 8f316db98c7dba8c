// rmhd_internal.h -- declarations shared by the translation units of the CUDA
// library (kernel launchers and plain-data parameter blocks). Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rmhd {

// Device layout of one field: variable planes of `plane` doubles each; cell
// (i, j) of variable v at base[v * plane + j * nx + i]. plane is nx * ny
// rounded up to 64 elements so every plane starts 512-byte aligned.
struct Grid {
    int nx, ny;
    int bcx, bcy;      // 0 outflow, 1 periodic
    long long ncell;   // nx * ny
    long long plane;
    double dx, dy;
    double rdx4, rdy4;  // 0.25 / dx, 0.25 / dy (host-computed)
    int nz, bcz;        // 3-D grids: cells and boundary condition along z (nz = 1: none)
    double dz, rdz4;
    // Index map of a flux tile: cell (i, j) of the tile's 2-D grid sits at
    // zoff * blockIdx.z + j * row + i (x-y planes: row = nx, zoff = nx ny;
    // x-z slabs of a 3-D grid: row = nx ny, zoff = nx).
    long long row, zoff;
    // Slab of a domain decomposed along y (2-D grids): the two rows below row
    // 0 (hlo) and above row ny - 1 (hhi) of every staged variable (the N_c
    // conserved, then the N_w internal primitives), [NC + NW][2][nx] each,
    // filled by halo exchange with the neighbouring slabs. Null on a side
    // without a neighbour: the boundary condition bcy applies there.
    const double *hlo, *hhi;
};

// Physical constants of a run plus host-precomputed reciprocals (the device
// avoids IEEE FP64 divisions, which cost ~7.5 FP64 ops each on GB300).
struct Phys {
    double gamma, sigma, kappa, mu_e, mu_p;
    double inv_dmu;  // 1 / (mu_e - mu_p)
    double eta;      // 1 / sigma
    double mur;      // max(|mu_e|, |mu_p|), scale of the two-fluid weighted unknowns
    double imur;     // 1 / mur
};

// One flux pass of an IMEX step (Eq. implicit stage / correction stage):
// L and Psi of the stage state are combined into nout (1-3) outputs, e.g. for
// SSP2(222) pass 1: r2 = q^n + dt L + (1 - 2 gamma) dt Psi and
// acc = q^n + dt/2 (L + Psi); pass 2: q^{n+1} = acc + dt/2 (L + Psi).
struct FluxArgs {
    const double *q;        // stage state, NC planes
    const double *w;        // stage primitives, NW planes
    const double *base[3];  // base of each output (may be the output itself: in-place update)
    double *out[3];         // out[k] = base[k] + cL[k] L + cS[k] Psi, k < nout
    double cL[3], cS[3];    // dt times the tableau coefficients (batches: per unit dt, scaled per run)
    double *wcarry;         // if not null: the stage primitives are copied here (next warm start)
    double *lout;           // nout = 0 (x-y pass of a 3-D grid): L_x + L_y is written here, nothing else
    const double *lin;      // if not null: added to L before the combinations (z pass of a 3-D grid)
    double *srcg;           // FP64 line-sweep passes: planes written by the stage kernel at the stage
                            // state: one fluid J (3), Z, p + (E^2+B^2)/2; two fluids Sbar (3), taubar, E (3)
    double *lscr;           // single fluid, FP64, 2-D: the x part of L between the x and y sweeps
                            // (NC planes of ncell cells)
};

struct StageArgs {
    const double *r;     // explicit part, NC planes
    const double *wwarm; // primitives used as the starting guess, NW planes
    double *q;           // stage solution, NC planes
    double *w;           // its primitives, NW planes
    int *status;
    double adt;          // a_ii dt
    unsigned long long *hist;  // if not null: per-solve histograms, FP32 Newton iterations [32], FP64 passes [8]
                               // and converged starts [4]
    int maxpass;               // cap on the FP64 refinement passes (0: the default, 8)
    // single fluid: cells whose first start failed, handed to the restart
    // kernel (rlist[0]: count, rlist[1]: restart blocks done, rlist[2 ..
    // rcap + 1]: cells; zero at creation, emptied by each restart kernel); a
    // cell beyond the capacity is reported as failed. Null: no restarts.
    int *rlist;
    int rcap;
    int first_start;  // tests of the restart path: 1 or 2 skips the earlier starts (0: all starts)
    // if not null, what the FP64 line-sweep flux pass takes from the stage
    // solve: one fluid, the current J, Z = rho h W^2 and p + (E^2 + B^2)/2 of
    // the stage state (5 planes); two fluids, its source entries Sbar (3),
    // taubar, E (3) (7 planes)
    double *src;
};

// Batched ensemble of independent 1-D runs packed one after another in every
// variable plane (run r occupies cells [offset[r], offset[r] + nx[r])).
struct BatchArgs {
    int nruns, nwork;
    const int2 *work;          // flux tiles: (run, first cell of the tile)
    const int *nx;             // cells per run
    const long long *offset;   // first packed cell of each run
    const double *dx, *dt;     // cell width and time step per run
    const double *rdx4;        // 0.25 / dx per run
    const double *sigma, *eta; // conductivity and 1/sigma per run
    const double *adt, *cpsi;  // a_ii dt and 1/(1 + a_ii dt kappa) per run
    const int *run_of;         // run of every packed cell
};

// launchers (return cudaGetLastError())
cudaError_t launch_stage(int model, const Grid &g, const Phys &ph, const StageArgs &a, cudaStream_t s);
cudaError_t launch_flux(int model, int precision, int nout, const Grid &g, const Phys &ph, const FluxArgs &a,
                        cudaStream_t s);
// 3-D grids: x-y pass into lbuf (L_x + L_y), then the z pass on x-z slabs
// adds L_z and forms the nout combinations of `a`.
cudaError_t launch_flux_3d(int model, int precision, int nout, const Grid &g, const Phys &ph, const FluxArgs &a,
                           double *lbuf, cudaStream_t s);
// primitives (user layout, device) -> conserved + internal primitives
cudaError_t launch_set_prims(int model, const Grid &g, const Phys &ph, const double *prims, double *q, double *w,
                             int *status, cudaStream_t s);
// internal state -> primitives in the user layout
cudaError_t launch_get_prims(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                             double *prims, cudaStream_t s);
// conserved -> internal primitives (recovery, cold start) into w; with prims
// set, also the primitives in the user layout (as launch_get_prims writes them)
cudaError_t launch_recover(int model, const Grid &g, const Phys &ph, const double *q, double *w, int *status,
                           cudaStream_t s, double *prims = nullptr);
// copy between the user layout [v][ny][nx] and the padded device layout
cudaError_t launch_pack(const Grid &g, int nvar, const double *user, double *dev, cudaStream_t s);
cudaError_t launch_unpack(const Grid &g, int nvar, const double *dev, double *user, cudaStream_t s);
// diagnostics: out[8] (see rmhd.h); partial sums in `scratch` (>= reduce_scratch_doubles())
size_t reduce_scratch_doubles();
cudaError_t launch_diagnostics(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                               double *scratch, double *out, cudaStream_t s);

// batched ensemble: stage solve per packed cell; flux tiles of width tile_x
// (64, 128 or 256) on `blocks` persistent CTAs; Gauss's law within each run
cudaError_t launch_stage_batch(int model, const Grid &g, const Phys &ph, const StageArgs &a, const BatchArgs &b,
                               int threads, cudaStream_t s);
cudaError_t launch_flux_batch(int model, int precision, int mode, const Grid &g, const Phys &ph, const FluxArgs &a,
                              const BatchArgs &b, int tile_x, int blocks, cudaStream_t s);
cudaError_t launch_set_prims_batch(int model, const Grid &g, const Phys &ph, const BatchArgs &b, const double *prims,
                                   double *q, double *w, int *status, cudaStream_t s);
// resident CTAs per SM of the batch flux kernel for a tile width (0 if unsupported)
int flux_batch_occupancy(int model, int precision, int tile_x);

// discrete adjoint (FP64; model 0 single fluid, 1 two fluids): one reverse
// step, the initial-map adjoint, and a deterministic plane sum
cudaError_t launch_adjoint_step(int model, const Grid &g, const Phys &ph, int scheme, double dt, const double *lam,
                                double *out, const double *const *Sq, const double *const *Sw, double *const *f,
                                double *const *fb, double *qbd, double *lq, double *lr2, double *lr3, double *sig,
                                cudaStream_t s);
cudaError_t launch_adjoint_prims(int model, const Grid &g, const Phys &ph, const double *q, const double *w,
                                 const double *lam, double *pbar, cudaStream_t s);
cudaError_t launch_sum(const double *x, long long n, double *out, cudaStream_t s);

inline int model_nc(int model) { return model == 0 ? 14 : 18; }
inline int model_nw(int model) { return model == 0 ? 5 : 10; }
inline int model_np(int model) { return model == 0 ? 11 : 16; }

} // namespace rmhd
