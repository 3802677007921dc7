// Internal interface between the C-ABI translation units: the mesh handle's
// layout, the element-kernel launcher and the error channel.  Not installed.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fem_b300.h"
#include "fem_plan.h"

namespace femi {
struct SolverWork;  // Newton-CG workspace, created on first use (fem_solver.cu)
struct LpMeshData;  // learned-preconditioner graph on the device (fem_learned.cu)
struct SparseData;  // sparse-K pattern, colouring and workspace (fem_sparse.cu)
struct AtomicData;  // element arrays of the atomic-scatter ablation (fem_atomic.cu)
struct NcmData;     // neural constitutive model: network and per-element arrays (fem_ncm.cu)
}

struct fem_mesh {
    fem::Plan plan;
    fem_mesh_info info{};
    int etype = 0, dim = 0, n_en = 0, precision = 0;
    bool per_elem_mat = false;
    double mu0 = 1.0, lam0 = 10.0;
    std::vector<void*> allocs;
    int64_t bytes = 0;
    // plan on the device
    int32_t* tile_round_ptr = nullptr;
    int64_t* tile_node_ptr = nullptr;
    int32_t* node_gid = nullptr;
    int32_t* node_slot = nullptr;
    uint8_t* round_nvalid = nullptr;
    int32_t* round_elem = nullptr;
    int32_t* slot_owner = nullptr;
    int4* shared_info = nullptr;  // per shared node: first slot, end slot, node, Dirichlet bits
    int32_t* orphans = nullptr;
    uint8_t* node_mask = nullptr;
    uint8_t* node_mask_local = nullptr;
    int max_nlp = 0;  // largest padded tile node count
    // element records per precision (index 0: FP64, 1: FP32)
    uint8_t* rec[2] = {nullptr, nullptr};
    int64_t rec_bytes[2] = {0, 0};
    int conn_bytes = 0;
    int stride = 0;
    void* X[2] = {nullptr, nullptr};
    // workspace
    void* partial = nullptr;
    double* tile_red = nullptr;
    unsigned* tile_counter = nullptr;
    int* status = nullptr;
    // Newton-CG workspace (allocated by the first fem_newton_step)
    femi::SolverWork* solver = nullptr;
    // host data of the learned preconditioner: the connectivity (its node
    // graph is built on first use) and per-node statistics (ln of the mean
    // incident mu, ln(mean lambda / mean mu), valence / 24)
    std::vector<int32_t> conn_host;
    std::vector<float> node_stats;
    femi::LpMeshData* lp = nullptr;
    // sparse K by colouring (built by the first fem_sparse_* call)
    femi::SparseData* sparse = nullptr;
    // host copies for the atomic-scatter ablation (natural element order)
    std::vector<double> coords_host, mu_host, lam_host;
    femi::AtomicData* atomic = nullptr;
    // neural constitutive model (set by fem_mesh_set_ncm; null: Neo-Hookean)
    femi::NcmData* ncm = nullptr;
    // stored linearisation per precision (OP_LINEARIZE; allocated on first use)
    void* lin[2] = {nullptr, nullptr};
    // pair records of the FP32 P1 pair kernels (mixed-precision P1 meshes):
    // records, first pair of every tile, and on the host the element of every
    // (pair, lane, half) slot (-1 empty) for moduli updates
    uint8_t* prec = nullptr;
    int prec_bytes = 0;
    int64_t n_pairs = 0;
    int32_t* tile_pair_ptr = nullptr;
    std::vector<int32_t> pair_elem;
};

namespace femi {
// records `msg` as the calling thread's last error and returns `s`
fem_status set_error(fem_status s, const std::string& msg);
// enqueue one element-kernel call (fem::Op `op`) on `st`; when `skip` is a
// device pointer, the kernels return at once if *skip is non-zero
// (vkv_tiles: for the HVP, leave the per-tile vKv partials in
// tile_partials(m) -- FP32 (hi, lo) pairs for FP32 calls, doubles for FP64,
// one per tile at a stride of 4 doubles -- for the caller to reduce).  The
// tile kernel and its finalize kernel are programmatic dependent launches.
fem_status run_op(fem_mesh* m, int dtype, int op, const void* u, const void* v, void* out,
                  double* out_scalar, unsigned flags, cudaStream_t st, const int* skip, int vkv_tiles = 0);
const double* tile_partials(const fem_mesh* m);
// frees the Newton-CG workspace of `m` (no-op without one)
void solver_free(fem_mesh* m);
// frees the learned-preconditioner data of `m` (no-op without it)
void lp_mesh_free(fem_mesh* m);
// frees the sparse-K data of `m` (no-op without it)
void sparse_free(fem_mesh* m);
// frees the atomic-ablation data of `m` (no-op without it)
void atomic_free(fem_mesh* m);
// the sparse pattern on the device (built on first use): CSR row pointers
// over DOFs, and the node lists N(n) as a node CSR (fem_sparse.cu)
fem_status sparse_arrays(fem_mesh* m, const int64_t** row_ptr, const int64_t** node_ptr, const int32_t** node_idx,
                         int64_t* nnz);
// neural constitutive model (fem_ncm.cu).  An internal flag of run_op /
// launch: the network's coefficients are current for this u and dtype (a
// PCG solve at a fixed state), so the coefficient pass is skipped.
constexpr unsigned kFlagNcmCurrent = 1u << 16;
// internal flag: an HVP at the state of the last OP_LINEARIZE call in this
// precision (Neo-Hookean P1 meshes): it reads the stored linearisation
constexpr unsigned kFlagUseLin = 1u << 17;
// internal: an energy call prepares the network's coefficients with their
// gradients too, so that a residual at the same state may follow with
// kFlagNcmCurrent (the Newton line search: energy at the trial point, then,
// once it is accepted, the residual there)
constexpr unsigned kFlagNcmGrad = 1u << 18;
void ncm_free(fem_mesh* m);
// allocates the per-element arrays of `dtype` on first use
fem_status ncm_prepare(fem_mesh* m, int dtype, cudaStream_t st);
// the network on every element's invariants: coefficients in record order
// (mode 0: value and scale, 1: also the gradient, 2: also the Hessian)
fem_status ncm_coefficients(fem_mesh* m, int dtype, int mode, cudaStream_t st, const int* skip);
const void* ncm_coef(const fem_mesh* m, int pi);
void* ncm_inv(const fem_mesh* m, int pi);
// P1 geometry of one element (vertices Xe [(D+1) * D]): grad N_a of the
// first D vertices (the last one is the reference) and w det J
void p1_geometry(int D, const double* Xe, double* out /* D * D + 1 */);
// fills the CG preconditioner blocks Minv [n_nodes * 9] (FP32) from the
// learned network `lp` at the FP32 state u: block diagonal, features,
// network, SPD map (fem_learned.cu)
fem_status lp_precondition(const void* lp, fem_mesh* m, const float* u, float* Minv, cudaStream_t st);
}  // namespace femi
