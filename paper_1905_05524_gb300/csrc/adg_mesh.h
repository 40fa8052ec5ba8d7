// Internal definition of the mesh object and shared host helpers of the
// library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "adg_internal.h"

struct adg_mesh {
    adg_mesh_desc d;
    int N = 0, n = 0, cells = 0;
    adg::Basis B;
    adg::Phys P;
    double* u = nullptr;
    double* rvol = nullptr;
    double* trace = nullptr;
    double* trace_bar = nullptr; // adjoint of the traces (allocated on first adg_step_adjoint)
    double* tv = nullptr;
    double* stats = nullptr;     // device [4]: mean, sigma; given mean, sigma (adg_tv_flags)
    double* part = nullptr;      // device TV statistics scratch: block triples and combine weights
    int tv_prep_cells = -1;      // cell count the combine weights in `part` were prepared for
    double* speed = nullptr;     // device partial maxima
    int speed_blocks = 0;
    int* flag = nullptr;         // device int
    double* bgbuf = nullptr;     // pbar_node, rhobar_node, pbar_face, rhobar_face
    adg::Background bg{};
    // mixed precision
    adg::BasisF Bf;
    adg::PhysF Pf;
    void* mixbuf = nullptr;
    adg::MixedBg mbg{};
    double t = 0.0;
    bool predicted = false;
    double pred_dt = 0.0;
    // adaptive 3:1 tree (desc.max_levels > 0); cells = number of leaves
    int amr = 0;
    void* tree = nullptr;         // host tree (adg_amr.cu)
    double* geo = nullptr;        // [leaves][4]: x0, y0, hx, hy of each leaf
    int* nbr = nullptr;           // [leaves][4 faces][5]: type, id0, id1, id2, sub-face
    double* bgl = nullptr;        // [leaves][n][2] node background, then [leaves][2][2] N/S faces
    double* mbl64 = nullptr;      // mixed precision: per-leaf FP64 background (adg_amr.cu upload_tables)
    float* mblf = nullptr;        // mixed precision: per-leaf FP32 background
    int leaf_cap = 0;             // leaves the per-leaf buffers and tables hold (grow-only)
    double* u_spare = nullptr;    // second state buffer: adaptation writes the new state here, then swaps
    int* dtrans = nullptr;        // [leaf_cap][12] transfer rules of an adaptation
    double hmin = 0.0;            // smallest leaf size (dt rule)
    double* halo = nullptr;       // strip decomposition: [2][nx][17][n] south, north halo traces
    unsigned epoch = 0;           // changes whenever the state or workspace buffers move (adg_adapt)
    // local time stepping (adg_step_lts): per-time-node traces and fine-flux sums, grow-only
    double* lts_ttrace = nullptr;
    double* lts_acc = nullptr;
    int lts_cap = 0;
};

namespace adg {
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
bool build_basis(int N, Basis& B);
int set_device(const adg_mesh* m);

// adaptive-mesh path (adg_amr.cu)
int amr_setup(adg_mesh* m);
void amr_free(adg_mesh* m);
int amr_predictor(adg_mesh* m, double dt, void* stream);
int amr_corrector(adg_mesh* m, double dt, void* stream);
int amr_tv_cells(adg_mesh* m, int var, double* tv, double* part, void* stream);
int amr_max_speed(adg_mesh* m, double* lam_max, void* stream);
int amr_init_scenario(adg_mesh* m, const adg_scenario* s, void* stream);
const void* amr_ops(const adg_mesh* m);
int amr_step_lts(adg_mesh* m, double dt, double* cycle, void* stream);
}  // namespace adg

#define ADG_CK(call, what)                                        \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return adg::cuda_fail(e_, what);   \
    } while (0)
