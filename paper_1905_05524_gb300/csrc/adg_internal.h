// Internal declarations shared by the translation units of libaderdg
// (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/aderdg.h"

namespace adg {

constexpr int kMaxN = ADG_MAX_DEGREE + 1;  // nodes per direction

// One-dimensional operators of the degree-N nodal Gauss-Legendre basis on
// [0, 1], passed to kernels by value (lands in the constant bank).
struct Basis {
    int n;
    double xi[kMaxN];         // nodes
    double w[kMaxN];          // weights, sum 1
    double phi0[kMaxN];       // phi_j(0)
    double phi1[kMaxN];       // phi_j(1)
    double D[kMaxN][kMaxN];   // D[i][j] = phi_j'(xi_i)
    double Kw[kMaxN][kMaxN];  // (K1^{-1})[l][k] * w_k  (time update of the predictor)
    double Kw1[kMaxN];        // sum_k Kw[l][k] (first sweep: time-constant residual)
    double Vx[kMaxN][kMaxN];  // Vx[p][i] = w_p D[p][i] / w_i (weak volume term)
    double lift0[kMaxN];      // phi_i(0) / w_i
    double lift1[kMaxN];      // phi_i(1) / w_i
};

// Physical and mesh constants of one mesh.
struct Phys {
    double gamma, gm1, R, invR, mu, kappa, g, cp, p0, theta0, Rcp;
    double lamv;              // max(4/3, gamma/Pr) * mu  (viscous eigenvalue * rho)
    double eta_x, eta_y;      // (2N+1) / (h sqrt(pi/2)) per direction
    double hx, hy, inv_hx, inv_hy, x0, y0;
    int gravity;
    int source;
    double sa, sL, sU, sp;    // steady manufactured source parameters
    int nx, ny, bc_x, bc_y;
    double lid_u = 0.0;       // ADG_BC_NOSLIP: x-velocity of the north wall
    int bc_field = 0;         // ADG_BC_ANALYTIC: ADG_FIELD_*
};

// Per-mesh device tables of the hydrostatic background (zero without gravity).
struct Background {
    const double* pbar_node;    // [ny][n]  at node heights y0 + (iy + xi_j) hy
    const double* rhobar_node;  // [ny][n]
    const double* pbar_face;    // [ny+1]   at face heights y0 + f hy
    const double* rhobar_face;  // [ny+1]
    const double* halo_s = nullptr;  // strip decomposition: north traces of the strip below [nx][17][n]
    const double* halo_n = nullptr;  // south traces of the strip above
};

// Trace record per face node: q-bar(4), normal flux(4), qx-bar(4), qy-bar(4), s(1)
constexpr int kTraceComps = 17;

// FP32 copies of the basis and constants for the mixed-precision kernels.
struct BasisF {
    float xi[kMaxN], w[kMaxN], phi0[kMaxN], phi1[kMaxN];
    float D[kMaxN][kMaxN], Kw[kMaxN][kMaxN], Kw1[kMaxN], Vx[kMaxN][kMaxN];
    float lift0[kMaxN], lift1[kMaxN];
};

struct PhysF {
    float gamma, gm1, R, invR, mu, kappa, g, cp, lamv, eta_x, eta_y;
    float hx, hy, inv_hx, inv_hy, x0, y0;
    float sa, sL, sU, sp;
    int gravity, source, nx, ny, bc_x, bc_y;
};

// Background tables of the mixed path (zero without gravity).  Node tables
// are indexed [iy * n + j]; face table [iy][0: north, 1: south][kFaceBg].
// Per y-face of a row: [0..2] rhobar, Ebar, pbar of the extrapolated nodal
// background (the base of the traces' perturbations); [3..5] the exact
// background at the face height (the slip-wall ghost state); [6..7] formed
// in FP64: on a wall face the exact minus the extrapolated rhobar and Ebar
// (the ghost's perturbation against the trace's base), on any other face
// the upper row's extrapolated rhobar, Ebar minus the lower row's (the two
// cells' bases differ there).
constexpr int kFaceBg = 8;
struct MixedBg {
    const double* rb;   // rhobar at nodes (FP64, for the perturbation split)
    const double* Eb;   // Ebar = pbar/(gamma-1) + rhobar g z at nodes (FP64)
    const float* pb;    // pbar at nodes
    const float* dzr;   // d rhobar/dz of the nodal interpolant
    const float* dzE;   // d Ebar/dz of the nodal interpolant
    const float* face;  // [ny][2][kFaceBg]
};

// One instance of a batched launch (device table entry) and one tile of
// consecutive cells of an instance.
struct MixedInst {
    double* u;
    float* rvol;
    float* trace;
    int cells;
    float dtf;
    double dt;
    PhysF P;
    MixedBg bg;
};
// Adaptive mixed-precision instance of a batch: the leaf predictor writes the
// FP64 residual and traces that the FP64 corrector with its hanging faces
// reads (adg_amr.cu); per-leaf geometry, neighbour and background tables.
struct AmrInst {
    double* u;
    double* rvol;
    double* trace;
    int cells;
    float dtf;
    double dt;
    PhysF Pf;
    Phys P;
    const double* geo;
    const int* nbr;
    const double* bgl;
    const double* mb64;
    const float* mbf;
};
// Uniform FP64 instance of a batch (the per-mesh FP64 bodies of adg_fp64.cu).
struct Fp64Inst {
    double* u;
    double* rvol;
    double* trace;
    int cells;
    double dt;
    Phys P;
    Background bg;
};
// A tile of a batch: inst >= 0 names a uniform instance, inst < 0 the
// adaptive instance -inst - 1; c0 is its first cell (leaf).
struct BatchTile {
    int inst, c0;
};
constexpr int kBatchCandidates = 4;  // predictor candidates the autotuner times (three tile sizes, node pairs)

// Kernel launchers (adg_fp64.cu, adg_mixed.cu, adg_tv.cu).  They return a
// cudaError_t value as int.
// Cells per block of the per-cell kernels (predictors, correctors, TV): one
// thread per node, whole warps as far as n^2 allows (N = 4: 5 cells = 125 of
// 128 lanes).  Every block that produces TV values also publishes the
// (count, mean, M2) triple of its cells, and the statistics combine these
// block triples.
constexpr int tv_cpb(int N) { return N == 1 ? 32 : N == 2 ? 16 : N == 3 ? 8 : N == 4 ? 5 : N == 5 ? 4 : 2; }
constexpr int kTvThreads = 256;  // threads per block of the statistics-and-flags kernel
constexpr int kTvLevels = 8;     // its combine tree: 5 levels within warps, 3 across the 8 warps

// Where the statistics kernel finds the block triples and the Chan weights
// of its fixed combine order (tv_stats_prepare).
struct TvStatsArgs {
    const double* part = nullptr;   // [3 * nblk] block triples (count, mean, M2)
    const double* wfold = nullptr;  // [2 * nblk] weights of the per-thread left folds
    const double* wtree = nullptr;  // [2 * kTvLevels * kTvThreads] weights of the tree over the threads
    int nblk = 0, per = 0, cells = 0;
};

// TV indicator evaluated by the corrector on the state it has just updated
// (the corrector launchers take nullptr for none).
struct TvEpilogue {
    double* tv = nullptr;            // [cells] output
    double* part = nullptr;          // [3 * tv_stats_blocks] block triples output
    int var = 0;                     // ADG_TV_THETA or ADG_TV_RHO
    double theta0 = 0.0, Rcp = 0.0;  // background potential temperature, R/c_p
};

int launch_predictor_fp64(int N, const double* u, double* rvol, double* trace, int cells,
                          double dt, double t, const Basis& B, const Phys& P,
                          const Background& bg, void* stream);
// t: time at the start of the step (analytic boundary data)
int launch_corrector_fp64(int N, double* u, const double* rvol, const double* trace, int cells,
                          double dt, const Basis& B, const Phys& P, const Background& bg,
                          void* stream, const TvEpilogue* epi = nullptr, double t = 0.0);
int launch_predictor_mixed(int N, const double* u, float* rvol, float* trace, int cells, double dt,
                           const BasisF& B, const PhysF& P, const MixedBg& bg, void* stream);
// the mixed predictor with its derivative contractions on the tensor cores
// (mma.sync TF32 with the three-term split, or BF16 operands split in three; adg_mixed_tc.cu), degrees 3, 5, 7
bool tc_degree_supported(int N);
int launch_predictor_mixed_tc(int N, const double* u, float* rvol, float* trace, int cells, double dt,
                              const BasisF& B, const PhysF& P, const MixedBg& bg, bool bf16, void* stream);
int launch_corrector_mixed(int N, double* u, const float* rvol, const float* trace, int cells,
                           double dt, const BasisF& B, const PhysF& P, const MixedBg& bg, void* stream,
                           const TvEpilogue* epi = nullptr);
// phase 0: predictor, 1: corrector.  tiles == nullptr: query -- returns the
// cells per block and writes the persistent grid size to *blocks_out; otherwise
// launches with the grid size in *blocks_out.
// Batched persistent launch over uniform FP64 instances (adg_fp64.cu); with
// tiles == NULL: query the cells per block and persistent grid.
int launch_batch_fp64(int N, int phase, const Fp64Inst* insts, const BatchTile* tiles, int ntiles, const Basis& B,
                      int* cpb_out, int* blocks_out, void* stream);
// Batched persistent launch over uniform (insts) and adaptive (ainsts, may be
// NULL) mixed-precision instances (adg_amr.cu).  B, ops: FP64 basis and the
// adaptive mesh's prolongation/restriction operators (used when ainsts is
// given).  With tiles == NULL: query the cells per block and persistent grid.
int launch_batch_mixed(int N, int cand, int phase, const MixedInst* insts, const AmrInst* ainsts,
                       const BatchTile* tiles, int ntiles, const BasisF& Bf, const Basis& B, const void* ops,
                       int* cpb_out, int* blocks_out, void* stream);
int launch_step_adjoint_fp64(int N, const double* u, const double* lam, double* lam_out, const double* trace,
                             double* trace_bar, int cells, double dt, const Basis& B, const Phys& P,
                             const Background& bg, void* stream);
// TV per cell, plus the (count, mean, M2) triple of every block's cells into part
int launch_tv_cells(int N, const double* u, double* tv, double* part, int cells, int var, const Basis& B,
                    const Phys& P, void* stream);
int launch_tv_cells_mixed(int N, const double* u, double* tv, double* part, int cells, int var,
                          const BasisF& B, const PhysF& P, const MixedBg& bg, double theta0, double Rcp,
                          void* stream);
// Statistics scratch `part`: [3 nblk] block triples | [2 nblk] fold weights |
// [2 kTvLevels kTvThreads] tree weights, nblk = tv_stats_blocks(N, cells).
int tv_stats_blocks(int N, int cells);
size_t tv_stats_scratch_doubles(int N, int cells);
// Chan weights of the combine order for (N, cells) into `part` (host
// division, one copy; synchronises `stream`); needed once per cell count.
int tv_stats_prepare(int N, int cells, double* part, void* stream);
TvStatsArgs tv_stats_args(int N, int cells, const double* part);
// mean and sigma from the block triples into stats_dev[0..1]; flags if not null
int launch_tv_stats_flags(const double* tv, const TvStatsArgs& st, double T_r, double T_c, double* stats_dev,
                          int8_t* flags, void* stream);
// flags from (mean, sigma) held in device memory at stats_dev
int launch_tv_flags_given(const double* tv, int cells, const double* stats_dev, double T_r, double T_c,
                          int8_t* flags, void* stream);
int launch_max_speed(int N, const double* u, double* partial, int cells, const Basis& B,
                     const Phys& P, int* nblocks_out, void* stream);
int launch_init_scenario(int N, double* u, int cells, int kind, double A, double a, double xc,
                         double zc, const Basis& B, const Phys& P, void* stream);
int launch_check_finite(const double* u, size_t count, int* flag, void* stream);

}  // namespace adg
