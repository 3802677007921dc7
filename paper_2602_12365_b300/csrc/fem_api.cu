// C ABI of the B300 FEM hot path: mesh handle, element kernels, status.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fem_b300.h"
#include "fem_internal.h"
#include "fem_kernels.cuh"
#include "fem_pair.cuh"

// the FP32 P1 residual and HVP through the pair kernels (0: the one-element
// tile kernels)
#ifndef FEM_PAIR_KERNELS
#define FEM_PAIR_KERNELS 1
#endif
#include "fem_plan.h"

static_assert(fem::kEmptyLane == fem::kNoNode, "kernel and planner agree on empty lanes");

namespace {
thread_local std::string g_err;

fem_status fail(fem_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(FEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
}  // namespace

namespace {

template <typename T>
fem_status upload(fem_mesh* m, T** dst, const T* src, size_t n, cudaStream_t st) {
    size_t bytes = sizeof(T) * (n > 0 ? n : 1);
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, bytes));
    m->allocs.push_back(p);
    m->bytes += (int64_t)bytes;
    if (src && n) CUDA_TRY(cudaMemcpyAsync(p, src, sizeof(T) * n, cudaMemcpyHostToDevice, st));
    *dst = static_cast<T*>(p);
    return FEM_OK;
}

fem_status zalloc(fem_mesh* m, void** dst, size_t bytes, cudaStream_t st) {
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, bytes > 0 ? bytes : 16));
    m->allocs.push_back(p);
    m->bytes += (int64_t)bytes;
    CUDA_TRY(cudaMemsetAsync(p, 0, bytes > 0 ? bytes : 16, st));
    *dst = p;
    return FEM_OK;
}

void free_all(fem_mesh* m) {
    for (void* p : m->allocs) cudaFree(p);
    m->allocs.clear();
}

int dim_of(int et) { return et == 0 ? 2 : 3; }
int nen_of(int et) { return et == 0 ? 3 : (et == 1 ? 4 : 8); }

// P1 shape-function gradients and w det J from the vertex positions:
// J = [X_1 - X_0, ..., X_D - X_0] (reference gradients of N_1..N_D are the
// unit vectors), grad N_a = row a-1 of J^-1 for a >= 1, grad N_0 = -sum.
bool p1_geometry(int D, const double* Xe, double (*g)[3], double* wdJ) {
    double J[3][3] = {{0}};
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) J[i][j] = Xe[(j + 1) * D + i] - Xe[i];
    double det, Ji[3][3];
    if (D == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
        *wdJ = det / 2.0;
    } else {
        double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        Ji[0][0] = c00 / det;
        Ji[1][0] = c01 / det;
        Ji[2][0] = c02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        *wdJ = det / 6.0;
    }
    if (!(det > 0.0)) return false;
    for (int k = 0; k < D; ++k) g[0][k] = 0.0;
    for (int a = 1; a <= D; ++a)
        for (int k = 0; k < D; ++k) {
            g[a][k] = Ji[a - 1][k];
            g[0][k] -= Ji[a - 1][k];
        }
    return true;
}

// det J of a Q1 element at every Gauss point must be positive
bool hex_positive(const double* Xe) {
    for (int q = 0; q < 8; ++q) {
        double J[3][3] = {{0}};
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] += Xe[a * 3 + i] * fem::hex_dN(a, q, j);
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0)) return false;
    }
    return true;
}

// Record of one round (one bulk copy): u16 conn[32][PAD] | T elem[32][stride],
// elem = (grad N_0 .. grad N_{NEN-2}, w det J | mu, lambda), stride even.
// scalars per element in a round record: P1 geometry (grad N of all but the
// last vertex, then w det J), then (mu, lambda) when they vary per element
int elem_stride(int etype, bool mat) {
    const int NG = etype == 0 ? 5 : (etype == 1 ? 10 : 0);
    return NG + (mat ? 2 : 0);
}

// P1 gradients and weight for the vertex order the kernel uses (any
// permutation of the element's vertices): grad N_a from the rows of J^-1,
// w det J from |det J| (an odd permutation flips the sign of det J).
}  // namespace

void femi::p1_geometry(int D, const double* Xe, double* out /* (NEN-1)*D + 1 */) {
    double g[4][3], wdJ;
    double J[3][3] = {{0}};
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) J[i][j] = Xe[(j + 1) * D + i] - Xe[i];
    double Ji[3][3], det;
    if (D == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
        wdJ = std::fabs(det) / 2.0;
    } else {
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        Ji[0][0] = c00 / det;
        Ji[1][0] = c01 / det;
        Ji[2][0] = c02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        wdJ = std::fabs(det) / 6.0;
    }
    for (int k = 0; k < D; ++k) g[0][k] = 0.0;
    for (int a = 1; a <= D; ++a)
        for (int k = 0; k < D; ++k) {
            g[a][k] = Ji[a - 1][k];
            g[0][k] -= Ji[a - 1][k];
        }
    // the kernel takes the LAST vertex as reference: store grad N_0..N_{D-1}
    for (int a = 0; a < D; ++a)
        for (int k = 0; k < D; ++k) out[a * D + k] = g[a][k];
    out[D * D] = wdJ;
}

namespace {

template <typename T>
void pack_records(fem_mesh* m, const fem_mesh_desc* d, std::vector<uint8_t>& out, int pi) {
    const fem::Plan& P = m->plan;
    const int D = m->dim;
    const int NG = m->etype == 0 ? 5 : (m->etype == 1 ? 10 : 0);
    const int conn_bytes = 2 * 32 * P.n_en_pad;
    const int stride = elem_stride(m->etype, m->per_elem_mat);
    const int64_t RB = conn_bytes + (int64_t)sizeof(T) * 32 * stride;
    m->rec_bytes[pi] = RB;
    m->conn_bytes = conn_bytes;
    m->stride = stride;
    out.assign((size_t)(P.n_rounds() * RB), 0);
    double Xe[4 * 3], geo[10];
    for (int t = 0; t < P.n_tiles(); ++t) {
        const int32_t* gid = P.node_gid.data() + P.tile_node_ptr[t];
        for (int64_t r = P.tile_round_ptr[t]; r < P.tile_round_ptr[t + 1]; ++r) {
            uint8_t* rec = out.data() + r * RB;
            std::memcpy(rec, P.round_conn.data() + r * 32 * P.n_en_pad, conn_bytes);
            // geometry in 16-byte chunks (CW scalars of every lane, lane-major),
            // then one (mu, lambda) pair per lane
            T* el0 = reinterpret_cast<T*>(rec + conn_bytes);
            constexpr int CW = 16 / (int)sizeof(T);
            for (int l = 0; l < P.round_nvalid[r]; ++l) {
                const int32_t e = P.round_elem[r * 32 + l];
                if (NG) {
                    const uint16_t* c = P.round_conn.data() + (r * 32 + l) * P.n_en_pad;
                    for (int a = 0; a <= D; ++a)
                        for (int k = 0; k < D; ++k) Xe[a * D + k] = d->coords[(size_t)gid[c[a]] * D + k];
                    femi::p1_geometry(D, Xe, geo);
                    for (int k = 0; k * CW < NG; ++k) {
                        const int w = std::min(CW, NG - k * CW);
                        for (int j = 0; j < w; ++j) el0[32 * k * CW + l * w + j] = (T)geo[k * CW + j];
                    }
                }
                if (m->per_elem_mat) {
                    el0[32 * NG + 2 * l + 0] = (T)d->mu[e];
                    el0[32 * NG + 2 * l + 1] = (T)d->lambda[e];
                }
            }
        }
    }
}

// Pair records of the FP32 P1 pair kernels (fem_pair.cuh): for every tile,
// warp by warp (warp w runs fem::pair_rounds(R, w) consecutive rounds of the
// tile's R), the warp's rounds two at a time: A = its 2k-th round, B = the
// next one or nothing.  Per lane: one 16-byte chunk of local node ids
// (A's NEN, padded to 4, then B's; a lane without an element names the dummy
// node `dummy`), the NG geometry values as (A, B) pairs in 16-byte chunks,
// and (mu_A, mu_B, lam_A, lam_B) when the moduli vary per element.  Returns
// the first pair of every tile in tile_pair_ptr.
void pack_pair_records(fem_mesh* m, const fem_mesh_desc* d, std::vector<uint8_t>& out,
                       std::vector<int32_t>& tile_pair_ptr, int dummy) {
    const fem::Plan& P = m->plan;
    const int D = m->dim;
    const int NG = m->etype == 0 ? 5 : 10;
    const int NCH = m->etype == 0 ? 3 : 5;
    const int RB = fem::pair_rec_bytes(m->etype, m->per_elem_mat);
    const int nt = P.n_tiles();
    tile_pair_ptr.assign((size_t)nt + 1, 0);
    for (int t = 0; t < nt; ++t) {
        const int R = P.tile_round_ptr[t + 1] - P.tile_round_ptr[t];
        tile_pair_ptr[t + 1] = tile_pair_ptr[t] + fem::pair_first(R, fem::kWarps);
    }
    out.assign((size_t)tile_pair_ptr[nt] * RB, 0);
    m->pair_elem.assign((size_t)tile_pair_ptr[nt] * 64, -1);
    double Xe[4 * 3], geo[10];
    for (int t = 0; t < nt; ++t) {
        const int32_t* gid = P.node_gid.data() + P.tile_node_ptr[t];
        const int R = P.tile_round_ptr[t + 1] - P.tile_round_ptr[t];
        int pr = tile_pair_ptr[t];
        int r = P.tile_round_ptr[t];
        for (int w = 0; w < fem::kWarps; ++w) {
            const int nw = fem::pair_rounds(R, w);
            for (int k = 0; k < nw; k += 2, ++pr) {
                uint8_t* rec = out.data() + (size_t)pr * RB;
                uint16_t* ids = reinterpret_cast<uint16_t*>(rec);
                float* geo0 = reinterpret_cast<float*>(rec + 512);
                float* mat = reinterpret_cast<float*>(rec + 512 * (1 + NCH));
                for (int h = 0; h < 2; ++h) {
                    const int64_t rr = r + k + h;
                    const bool have_round = k + h < nw;
                    for (int l = 0; l < 32; ++l) {
                        const bool valid = have_round && l < P.round_nvalid[rr];
                        for (int a = 0; a < 4; ++a)
                            ids[l * 8 + h * 4 + a] =
                                (valid && a < m->n_en) ? P.round_conn[(rr * 32 + l) * P.n_en_pad + a] : (uint16_t)dummy;
                        if (!valid) continue;  // zero geometry and moduli
                        const int32_t e = P.round_elem[rr * 32 + l];
                        m->pair_elem[(size_t)pr * 64 + l * 2 + h] = e;
                        const uint16_t* c = P.round_conn.data() + (rr * 32 + l) * P.n_en_pad;
                        for (int a = 0; a <= D; ++a)
                            for (int q = 0; q < D; ++q) Xe[a * D + q] = d->coords[(size_t)gid[c[a]] * D + q];
                        femi::p1_geometry(D, Xe, geo);
                        // pair j of lane l: chunk j / 2, slot 2 (j % 2) + h
                        for (int j = 0; j < NG; ++j) geo0[(j / 2) * 128 + l * 4 + 2 * (j % 2) + h] = (float)geo[j];
                        if (m->per_elem_mat) {
                            mat[l * 4 + h] = (float)d->mu[e];
                            mat[l * 4 + 2 + h] = (float)d->lambda[e];
                        }
                    }
                }
            }
            r += nw;
        }
    }
}

using KFn = void (*)(const fem::KParams);

template <int ET, typename T>
KFn pick(int op) {
    switch (op) {
        case fem::OP_ENERGY: return fem::tile_kernel<ET, T, fem::OP_ENERGY>;
        case fem::OP_RESIDUAL: return fem::tile_kernel<ET, T, fem::OP_RESIDUAL>;
        case fem::OP_HVP: return fem::tile_kernel<ET, T, fem::OP_HVP>;
        case fem::OP_BLOCKDIAG: return fem::tile_kernel<ET, T, fem::OP_BLOCKDIAG>;
        default: return fem::tile_kernel<ET, T, fem::OP_PVJP>;
    }
}

// the neural constitutive model's kernels (P1 only)
template <int ET, typename T>
KFn pick_ncm(int op) {
    switch (op) {
        case fem::OP_ENERGY: return fem::tile_kernel<ET, T, fem::OP_ENERGY, true>;
        case fem::OP_RESIDUAL: return fem::tile_kernel<ET, T, fem::OP_RESIDUAL, true>;
        case fem::OP_HVP: return fem::tile_kernel<ET, T, fem::OP_HVP, true>;
        case fem::OP_BLOCKDIAG: return fem::tile_kernel<ET, T, fem::OP_BLOCKDIAG, true>;
        default: return fem::tile_kernel<ET, T, fem::OP_NCM_INV>;
    }
}

KFn pair_kernel_for(int et, int op, bool lin) {
    if (op == fem::OP_HVP && lin)
        return et == 0 ? fem::pair_kernel<0, fem::OP_HVP, true> : fem::pair_kernel<1, fem::OP_HVP, true>;
    if (op == fem::OP_HVP) return et == 0 ? fem::pair_kernel<0, fem::OP_HVP> : fem::pair_kernel<1, fem::OP_HVP>;
    if (op == fem::OP_LINEARIZE)
        return et == 0 ? fem::pair_kernel<0, fem::OP_LINEARIZE> : fem::pair_kernel<1, fem::OP_LINEARIZE>;
    return et == 0 ? fem::pair_kernel<0, fem::OP_RESIDUAL> : fem::pair_kernel<1, fem::OP_RESIDUAL>;
}

KFn kernel_for(int et, int dtype, int op, bool ncm, bool lin = false) {
    if (lin) {
        if (dtype == FEM_F64)
            return et == 0   ? fem::tile_kernel<0, double, fem::OP_HVP, false, true>
                   : et == 1 ? fem::tile_kernel<1, double, fem::OP_HVP, false, true>
                             : fem::tile_kernel<2, double, fem::OP_HVP, false, true>;
        return et == 0 ? fem::tile_kernel_lin<0>
                       : (et == 1 ? fem::tile_kernel_lin<1> : fem::tile_kernel_hex<fem::OP_HVP, true>);
    }
    if (op == fem::OP_LINEARIZE) {
        if (dtype == FEM_F64)
            return et == 0   ? fem::tile_kernel<0, double, fem::OP_LINEARIZE>
                   : et == 1 ? fem::tile_kernel<1, double, fem::OP_LINEARIZE>
                             : fem::tile_kernel<2, double, fem::OP_LINEARIZE>;
        return et == 0   ? fem::tile_kernel<0, float, fem::OP_LINEARIZE>
               : et == 1 ? fem::tile_kernel<1, float, fem::OP_LINEARIZE>
                         : fem::tile_kernel_hex<fem::OP_LINEARIZE>;
    }
    if (ncm || op == fem::OP_NCM_INV) {
        if (dtype == FEM_F64) return et == 0 ? pick_ncm<0, double>(op) : pick_ncm<1, double>(op);
        return et == 0 ? pick_ncm<0, float>(op) : pick_ncm<1, float>(op);
    }
    if (dtype == FEM_F64) {
        if (et == 0) return pick<0, double>(op);
        if (et == 1) return pick<1, double>(op);
        return pick<2, double>(op);
    }
    if (et == 0) return pick<0, float>(op);
    if (et == 1) return pick<1, float>(op);
    switch (op) {
        case fem::OP_ENERGY: return fem::tile_kernel_hex<fem::OP_ENERGY>;
        case fem::OP_RESIDUAL: return fem::tile_kernel_hex<fem::OP_RESIDUAL>;
        case fem::OP_HVP: return fem::tile_kernel_hex<fem::OP_HVP>;
        case fem::OP_BLOCKDIAG: return fem::tile_kernel_hex<fem::OP_BLOCKDIAG>;
        default: return fem::tile_kernel_hex<fem::OP_PVJP>;
    }
}

int max_optin_smem() {
    static int v = -1;
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 227 * 1024;
    }
    return v;
}

int record_bytes(int et, bool mat, int tsize) {
    const int pad = et == 2 ? 8 : 4;
    return 2 * 32 * pad + tsize * 32 * elem_stride(et, mat);
}

int max_padded_nodes(const fem::Plan& P) {
    int64_t w = 0;
    for (int t = 0; t < P.n_tiles(); ++t) w = std::max(w, P.tile_node_ptr[t + 1] - P.tile_node_ptr[t]);
    return (int)w;
}

int worst_smem(int et, int nlp, bool mixed, bool mat) {
    int w = 0;
    for (int op = 0; op < 5; ++op) {
        w = std::max(w, fem::smem_layout(et, 8, op, nlp, record_bytes(et, mat, 8)).total);
        if (mixed) w = std::max(w, fem::smem_layout(et, 4, op, nlp, record_bytes(et, mat, 4)).total);
    }
    // the HVP from a stored linearisation, and the pass that stores it
    w = std::max(w, fem::smem_layout(et, 8, fem::OP_HVP, nlp, record_bytes(et, mat, 8), true).total);
    w = std::max(w, fem::smem_layout(et, 8, fem::OP_LINEARIZE, nlp, record_bytes(et, mat, 8)).total);
    if (mixed) {
        w = std::max(w, fem::smem_layout(et, 4, fem::OP_HVP, nlp, record_bytes(et, mat, 4), true).total);
        w = std::max(w, fem::smem_layout(et, 4, fem::OP_LINEARIZE, nlp, record_bytes(et, mat, 4)).total);
    }
    return w;
}

template <int D, typename T>
KFn pick_fin(int op) {
    switch (op) {
        case fem::OP_RESIDUAL: return fem::finalize_kernel<D, T, fem::OP_RESIDUAL>;
        case fem::OP_HVP: return fem::finalize_kernel<D, T, fem::OP_HVP>;
        default: return fem::finalize_kernel<D, T, fem::OP_BLOCKDIAG>;
    }
}

KFn finalize_for(int dim, int dtype, int op) {
    if (dtype == FEM_F64) return dim == 2 ? pick_fin<2, double>(op) : pick_fin<3, double>(op);
    return dim == 2 ? pick_fin<2, float>(op) : pick_fin<3, float>(op);
}

// Module-scope scratch of fem_energy_static: one 256-byte line holding the
// energy reduction's arrival counter, then FEM_STATIC_MAX_TILES tile partials
// of 4 doubles.  One copy per device and process, zero at module load.
constexpr size_t kStaticCounterBytes = 256;
constexpr size_t kStaticScratchBytes = kStaticCounterBytes + (size_t)FEM_STATIC_MAX_TILES * 4 * sizeof(double);
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct ReductionScratch {
    double* tile_red;
    unsigned* counter;
};

// Device address of g_static_scratch in the current context.  The address
// is looked up (cudaGetSymbolAddress, with the context's device current) the
// first time a context calls, and cached keyed by the context handle, not by
// the device ordinal: after a device reset or a primary-context teardown the
// module is loaded again, the array may move, and the new context gets a
// fresh lookup instead of a stale pointer.
using CtxGetCurrentFn = int (*)(void**);  // cuCtxGetCurrent (CUresult, CUcontext*)

fem_status current_context(void** ctx) {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    *ctx = nullptr;
    if (!fn) return fail(FEM_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
    if (fn(ctx) != 0 || !*ctx) return fail(FEM_ERR_CUDA, "no current CUDA context for the static scratch");
    return FEM_OK;
}

fem_status static_scratch(ReductionScratch* out) {
    static std::mutex mu;
    static std::vector<std::pair<void*, void*>> addr;  // (context, device address)
    auto lookup = [](void** a) -> fem_status {
        const cudaError_t e = cudaGetSymbolAddress(a, g_static_scratch);
        if (e != cudaSuccess || !*a)
            return fail(FEM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                          cudaGetErrorString(e));
        return FEM_OK;
    };
    void* ctx = nullptr;
    void* a = nullptr;
    fem_status cs = current_context(&ctx);
    if (cs != FEM_OK) {
        // no context is current on this thread yet: the lookup makes the
        // device's primary context current; then ask again
        if ((cs = lookup(&a)) != FEM_OK || (cs = current_context(&ctx)) != FEM_OK) return cs;
    }
    std::lock_guard<std::mutex> lk(mu);
    bool cached = false;
    for (const auto& e : addr)
        if (e.first == ctx) a = e.second, cached = true;
    if (!cached) {
        if (!a && (cs = lookup(&a)) != FEM_OK) return cs;
        addr.emplace_back(ctx, a);
    }
    unsigned char* base = static_cast<unsigned char*>(a);
    out->counter = reinterpret_cast<unsigned*>(base);
    out->tile_red = reinterpret_cast<double*>(base + kStaticCounterBytes);
    return FEM_OK;
}

fem_status launch(fem_mesh* m, int dtype, int op, const void* u, const void* v, void* out,
                  double* out_scalar, double* out_mu, double* out_lam, unsigned flags,
                  cudaStream_t st, const ReductionScratch* scratch = nullptr, const int* skip = nullptr,
                  int vkv_tiles = 0) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    if (dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    const int pi = dtype == FEM_F64 ? 0 : 1;
    const int tsize = dtype == FEM_F64 ? 8 : 4;
    // neural constitutive model: the network's coefficients at u (invariants
    // pass, then the network), unless the caller knows they are current
    const bool ncm = m->ncm != nullptr &&
                     (op == fem::OP_ENERGY || op == fem::OP_RESIDUAL || op == fem::OP_HVP || op == fem::OP_BLOCKDIAG);
    if (ncm && !(flags & femi::kFlagNcmCurrent)) {
        fem_status s = femi::ncm_prepare(m, dtype, st);
        if (s == FEM_OK)
            s = launch(m, dtype, fem::OP_NCM_INV, u, nullptr, nullptr, nullptr, nullptr, nullptr, 0, st, nullptr, skip,
                       0);
        const int mode = op == fem::OP_ENERGY ? ((flags & femi::kFlagNcmGrad) ? 1 : 0) : (op == fem::OP_RESIDUAL ? 1 : 2);
        if (s == FEM_OK) s = femi::ncm_coefficients(m, dtype, mode, st, skip);
        if (s != FEM_OK) return s;
    }
    flags &= ~(femi::kFlagNcmCurrent | femi::kFlagNcmGrad);
    // the stored linearisation: written by OP_LINEARIZE, read by an HVP that
    // asks for it (Neo-Hookean; per element for P1, per Gauss point for Q1)
    const bool lin = op == fem::OP_HVP && (flags & femi::kFlagUseLin) && !ncm;
    flags &= ~femi::kFlagUseLin;
    // FP32 P1 (Neo-Hookean, the handle's own workspace): the pair kernels for
    // the residual, the HVP (at u, or from the stored linearisation, which
    // the pair linearisation pass writes in pair-record order) and the
    // linearisation itself; an HVP with the last-CTA vKv total stays on the
    // tile kernel
    const bool pair_ok = FEM_PAIR_KERNELS && dtype == FEM_F32 && m->prec != nullptr && !ncm && scratch == nullptr;
    const bool pair = pair_ok && (op == fem::OP_RESIDUAL || op == fem::OP_LINEARIZE ||
                                  (op == fem::OP_HVP && out_scalar == nullptr));
    if (lin && pair_ok && !pair)
        return fail(FEM_ERR_ARG, "the FP32 stored linearisation serves HVPs without a vKv total");
    if (op == fem::OP_LINEARIZE) {
        if (m->ncm) return fail(FEM_ERR_ARG, "the stored linearisation covers the Neo-Hookean law");
        if (!m->lin[pi]) {
            void* q = nullptr;
            const size_t per_elem = m->etype == 2 ? 8 * fem::kHexLinVals : fem::kLinVals;
            size_t bytes = (size_t)m->plan.n_rounds() * 32 * per_elem * tsize;
            if (pair_ok) bytes = std::max(bytes, (size_t)m->n_pairs * fem::pair_lin_bytes(m->etype));
            fem_status s = zalloc(m, &q, bytes, st);
            if (s != FEM_OK) return s;
            m->lin[pi] = q;
        }
    }
    if (lin && !m->lin[pi]) return fail(FEM_ERR_ARG, "HVP from a linearisation that was never stored");
    fem::KParams p{};
    p.tile_round_ptr = m->tile_round_ptr;
    p.tile_node_ptr = m->tile_node_ptr;
    p.node_gid = m->node_gid;
    p.node_slot = m->node_slot;
    p.round_nvalid = m->round_nvalid;
    p.round_elem = m->round_elem;
    p.rec = m->rec[pi];
    p.rec_bytes = (int)m->rec_bytes[pi];
    p.conn_bytes = m->conn_bytes;
    p.stride = m->stride;
    p.has_mat = m->per_elem_mat ? 1 : 0;
    p.slot_owner = m->slot_owner;
    p.shared_info = m->shared_info;
    p.n_shared = (int)m->plan.shared_gid.size();
    p.orphans = m->orphans;
    p.n_orphans = (int)m->plan.orphans.size();
    p.node_mask = m->node_mask;
    p.node_mask_local = m->node_mask_local;
    p.max_nlp = m->max_nlp;
    p.X = m->X[pi];
    p.n_tiles = m->plan.n_tiles();
    p.mu0 = m->mu0;
    p.lam0 = m->lam0;
    p.partial = m->partial;
    p.tile_red = scratch ? scratch->tile_red : m->tile_red;
    p.tile_counter = scratch ? scratch->counter : m->tile_counter;
    p.status = m->status;
    p.skip = skip;
    p.vkv_tiles = vkv_tiles;
    if (m->ncm) {
        p.ncm_coef = femi::ncm_coef(m, pi);
        p.ncm_inv = femi::ncm_inv(m, pi);
    }
    p.lin = m->lin[pi];
    p.u = u;
    p.v = v;
    p.out = out;
    p.out_scalar = out_scalar;
    p.out_mu = out_mu;
    p.out_lam = out_lam;
    p.flags = flags;
    p.prec = m->prec;
    p.prec_bytes = m->prec_bytes;
    p.tile_pair_ptr = m->tile_pair_ptr;
    const int smem =
        pair ? fem::pair_layout(m->etype, op, lin, m->max_nlp, fem::pair_copy_bytes(m->etype, m->per_elem_mat, lin)).total
             : fem::smem_layout(m->etype, tsize, op, m->max_nlp, (int)m->rec_bytes[pi], lin).total;
    KFn fn = pair ? pair_kernel_for(m->etype, op, lin) : kernel_for(m->etype, dtype, op, ncm, lin);
    int grid = 0;
    {
        // raise the dynamic shared-memory limit once per (device, kernel)
        static std::mutex mu;
        static std::map<std::pair<int, const void*>, int> set_to;
        int dev = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(mu);
        auto key = std::make_pair(dev, reinterpret_cast<const void*>(fn));
        auto it = set_to.find(key);
        if (it == set_to.end() || it->second < smem) {
            CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            set_to[key] = smem;
        }
        // persistent grid: every resident slot, at most max_tiles_per_cta tiles each
        static std::map<std::pair<std::pair<int, const void*>, int>, int> resident;
        auto rk = std::make_pair(key, smem);
        auto ri = resident.find(rk);
        if (ri == resident.end()) {
            int per_sm = 0, sms = 0;
            CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, fem::kThreads, smem));
            CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            ri = resident.emplace(rk, std::max(1, per_sm) * sms).first;
        }
        grid = std::min(p.n_tiles, ri->second);
        const int cap = pair ? fem::kMaxTilesPerCta : fem::max_tiles_per_cta(m->etype);
        grid = std::max(grid, (p.n_tiles + cap - 1) / cap);
    }
    {
        // programmatic dependent launch: the CTAs are placed as the previous
        // kernel's blocks exit and wait on griddepcontrol.wait before their
        // first access to anything an earlier kernel writes
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(fem::kThreads);
        cfg.dynamicSmemBytes = (size_t)smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, p));
    }
    if (op == fem::OP_RESIDUAL || op == fem::OP_HVP || op == fem::OP_BLOCKDIAG) {
        // shared nodes: programmatic dependent launch, so the launch overlaps
        // the tile kernel's tail; the kernel waits on griddepcontrol.wait
        const int total = p.n_shared + p.n_orphans;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)std::max(1, (total + fem::kFinThreads - 1) / fem::kFinThreads));
        cfg.blockDim = dim3(fem::kFinThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CUDA_TRY(cudaLaunchKernelEx(&cfg, finalize_for(m->dim, dtype, op), p));
    }
    return FEM_OK;
}

fem_status plan_from_desc(const fem_mesh_desc* d, fem::Plan& plan, int tile_elems) {
    if (!d) return fail(FEM_ERR_ARG, "null descriptor");
    if (d->elem_type < 0 || d->elem_type > 2) return fail(FEM_ERR_ARG, "elem_type must be 0, 1 or 2");
    if (d->n_nodes <= 0 || d->n_elems <= 0) return fail(FEM_ERR_ARG, "empty mesh");
    if (!d->coords || !d->conn) return fail(FEM_ERR_ARG, "coords and conn are required");
    if ((d->mu == nullptr) != (d->lambda == nullptr))
        return fail(FEM_ERR_ARG, "mu and lambda must both be given or both be NULL");
    fem::MeshInput in;
    in.elem_type = d->elem_type;
    in.dim = dim_of(d->elem_type);
    in.n_en = nen_of(d->elem_type);
    in.n_nodes = d->n_nodes;
    in.n_el = d->n_elems;
    in.X = d->coords;
    in.conn = d->conn;
    in.tile_elems = tile_elems;
    std::string err = fem::build_plan(in, plan);
    if (!err.empty()) return fail(err.find("out of range") != std::string::npos ? FEM_ERR_ARG : FEM_ERR_BADMESH, err);
    return FEM_OK;
}

void fill_info(const fem::Plan& P, fem_mesh_info* info) {
    std::memset(info, 0, sizeof *info);
    info->n_nodes = P.n_nodes;
    info->n_elems = P.n_el;
    info->dim = P.dim;
    info->n_en = P.n_en;
    info->n_tiles = P.n_tiles();
    info->max_tile_nodes = P.max_tile_nodes;
    info->n_rounds = P.n_rounds();
    info->max_rounds = P.max_rounds;
    info->n_shared = (int32_t)P.shared_gid.size();
    info->n_slots = P.n_slots();
    info->n_local_nodes = (int64_t)P.node_gid.size();
    info->n_orphans = (int64_t)P.orphans.size();
    info->round_fill = P.n_rounds() ? (double)P.n_el / (32.0 * (double)P.n_rounds()) : 0.0;
}

}  // namespace

namespace femi {
fem_status set_error(fem_status s, const std::string& msg) { return fail(s, msg); }

fem_status run_op(fem_mesh* m, int dtype, int op, const void* u, const void* v, void* out,
                  double* out_scalar, unsigned flags, cudaStream_t st, const int* skip, int vkv_tiles) {
    return launch(m, dtype, op, u, v, out, out_scalar, nullptr, nullptr, flags, st, nullptr, skip, vkv_tiles);
}

const double* tile_partials(const fem_mesh* m) { return m->tile_red; }
}  // namespace femi

extern "C" {

const char* fem_last_error(void) { return g_err.c_str(); }

fem_status fem_plan_partition(const fem_mesh_desc* desc, int32_t* elem_tile, int64_t* elem_round,
                              int32_t* elem_lane, int32_t* elem_nodes, fem_mesh_info* info) {
    fem::Plan P;
    fem_status s = plan_from_desc(desc, P, desc ? desc->tile_elems : 0);
    if (s != FEM_OK) return s;
    for (int t = 0; t < P.n_tiles(); ++t)
        for (int32_t r = P.tile_round_ptr[t]; r < P.tile_round_ptr[t + 1]; ++r)
            for (int l = 0; l < P.round_nvalid[r]; ++l) {
                int32_t e = P.round_elem[(int64_t)r * 32 + l];
                if (elem_tile) elem_tile[e] = t;
                if (elem_round) elem_round[e] = r;
                if (elem_lane) elem_lane[e] = l;
                if (elem_nodes)
                    for (int a = 0; a < P.n_en; ++a)
                        elem_nodes[(int64_t)e * P.n_en + a] =
                            P.node_gid[P.tile_node_ptr[t] + P.round_conn[((int64_t)r * 32 + l) * P.n_en_pad + a]];
            }
    if (info) fill_info(P, info);
    return FEM_OK;
}

fem_status fem_mesh_create(const fem_mesh_desc* d, fem_mesh** out, void* stream) {
    if (!out) return fail(FEM_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!d) return fail(FEM_ERR_ARG, "null descriptor");
    if (d->precision != FEM_PREC_FP64 && d->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "precision must be FEM_PREC_FP64 or FEM_PREC_MIXED");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fem_mesh* m = new fem_mesh();
    m->etype = d->elem_type;
    m->precision = d->precision;
    m->dim = dim_of(d->elem_type);
    m->n_en = nen_of(d->elem_type);
    m->per_elem_mat = d->mu != nullptr;
    m->mu0 = d->mu0;
    m->lam0 = d->lambda0;
    const bool mixed = d->precision == FEM_PREC_MIXED;
    if (d->n_nodes > 0 && d->n_elems > 0 && d->conn) {
        // host data of the learned preconditioner (one pass over the elements)
        const int ne_n = nen_of(d->elem_type);
        m->conn_host.assign(d->conn, d->conn + d->n_elems * ne_n);
        if (d->coords) m->coords_host.assign(d->coords, d->coords + d->n_nodes * dim_of(d->elem_type));
        if (d->mu && d->lambda) {
            m->mu_host.assign(d->mu, d->mu + d->n_elems);
            m->lam_host.assign(d->lambda, d->lambda + d->n_elems);
        }
        std::vector<double> smu((size_t)d->n_nodes, 0.0), slam((size_t)d->n_nodes, 0.0), val((size_t)d->n_nodes, 0.0);
        for (int64_t e = 0; e < d->n_elems; ++e)
            for (int a = 0; a < ne_n; ++a) {
                const int32_t n = d->conn[e * ne_n + a];
                if (n < 0 || n >= d->n_nodes) continue;  // rejected by the planner below
                smu[n] += d->mu ? d->mu[e] : d->mu0;
                slam[n] += d->lambda ? d->lambda[e] : d->lambda0;
                val[n] += 1.0;
            }
        m->node_stats.resize((size_t)d->n_nodes * 3);
        for (int64_t n = 0; n < d->n_nodes; ++n) {
            const double mb = val[n] > 0 ? smu[n] / val[n] : d->mu0;
            const double lb = val[n] > 0 ? slam[n] / val[n] : d->lambda0;
            m->node_stats[n * 3 + 0] = (float)std::log(mb);
            m->node_stats[n * 3 + 1] = (float)std::log(lb / mb);
            m->node_stats[n * 3 + 2] = (float)(val[n] / 24.0);
        }
    }
    // plan; halve the tile until its shared memory fits the device
    int tile = d->tile_elems;
    fem_status s;
    for (int attempt = 0;; ++attempt) {
        s = plan_from_desc(d, m->plan, tile);
        if (s != FEM_OK) {
            delete m;
            return s;
        }
        if (worst_smem(m->etype, max_padded_nodes(m->plan), mixed, m->per_elem_mat) <= max_optin_smem()) break;
        tile = m->plan.tile_elems / 2;
        if (tile < 32 || attempt > 6) {
            delete m;
            return fail(FEM_ERR_BADMESH, "a tile's nodes do not fit in shared memory");
        }
    }
    const fem::Plan& P = m->plan;
    const int D = m->dim, NEN = m->n_en;
    const int64_t NE = d->n_elems, NN = d->n_nodes;

    // orientation checks in the input vertex order
    if (m->etype != 2) {
        double Xe[4 * 3], g[4][3], wdJ;
        for (int64_t e = 0; e < NE; ++e) {
            for (int a = 0; a < NEN; ++a)
                for (int k = 0; k < D; ++k) Xe[a * D + k] = d->coords[(size_t)d->conn[e * NEN + a] * D + k];
            if (!p1_geometry(D, Xe, g, &wdJ)) {
                delete m;
                return fail(FEM_ERR_BADMESH, "element " + std::to_string(e) + " has det J <= 0");
            }
        }
    } else {
        double Xe[24];
        for (int64_t e = 0; e < NE; ++e) {
            for (int a = 0; a < 8; ++a)
                for (int k = 0; k < 3; ++k) Xe[a * 3 + k] = d->coords[(size_t)d->conn[e * 8 + a] * 3 + k];
            if (!hex_positive(Xe)) {
                delete m;
                return fail(FEM_ERR_BADMESH, "hexahedron " + std::to_string(e) + " has det J <= 0");
            }
        }
    }
    std::vector<uint8_t> mask(NN, 0);
    if (d->dirichlet)
        for (int64_t n = 0; n < NN; ++n)
            for (int k = 0; k < D; ++k)
                if (d->dirichlet[n * D + k]) mask[n] |= (uint8_t)(1u << k);

#define UP(dst, vec) \
    if ((s = upload(m, &m->dst, (vec).data(), (vec).size(), st)) != FEM_OK) goto fail_out
    UP(tile_round_ptr, P.tile_round_ptr);
    UP(tile_node_ptr, P.tile_node_ptr);
    UP(node_gid, P.node_gid);
    UP(node_slot, P.node_slot);
    UP(round_nvalid, P.round_nvalid);
    UP(round_elem, P.round_elem);
    UP(slot_owner, P.slot_owner);
    {
        // one 16-byte record per shared node, so that the finalize kernel
        // issues its slot loads after a single load
        std::vector<int4> info(P.shared_gid.size());
        for (size_t j = 0; j < info.size(); ++j)
            info[j] = make_int4((int)P.shared_slot_ptr[j], (int)P.shared_slot_ptr[j + 1], P.shared_gid[j],
                                (int)mask[P.shared_gid[j]]);
        UP(shared_info, info);
    }
    UP(orphans, P.orphans);
    UP(node_mask, mask);
    {
        std::vector<uint8_t> mloc(P.node_gid.size(), 0);
        for (size_t j = 0; j < mloc.size(); ++j)
            if (P.node_gid[j] >= 0) mloc[j] = mask[P.node_gid[j]];
        UP(node_mask_local, mloc);
    }
    m->max_nlp = max_padded_nodes(P);
#undef UP
    {
        std::vector<uint8_t> recs;
        for (int pi = 0; pi < 2; ++pi) {
            if (pi == 1 && !mixed) break;
            if (pi == 0)
                pack_records<double>(m, d, recs, 0);
            else
                pack_records<float>(m, d, recs, 1);
            if ((s = upload(m, &m->rec[pi], recs.data(), recs.size(), st)) != FEM_OK) goto fail_out;
            if (m->etype == 2) {
                if (pi == 0) {
                    double* x = nullptr;
                    if ((s = upload(m, &x, d->coords, (size_t)NN * 3, st)) != FEM_OK) goto fail_out;
                    m->X[0] = x;
                } else {
                    std::vector<float> xf((size_t)NN * 3);
                    for (size_t i = 0; i < xf.size(); ++i) xf[i] = (float)d->coords[i];
                    float* x = nullptr;
                    if ((s = upload(m, &x, xf.data(), xf.size(), st)) != FEM_OK) goto fail_out;
                    m->X[1] = x;
                }
            }
            // records are host temporaries: finish the copy before reuse
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                s = fail(FEM_ERR_CUDA, "cudaStreamSynchronize failed during upload");
                goto fail_out;
            }
        }
    }
    if (mixed && m->etype < 2 && m->max_nlp < 0xFFFF) {
        // pair records of the FP32 pair kernels (the dummy node is max_nlp)
        std::vector<uint8_t> precs;
        std::vector<int32_t> tpp;
        pack_pair_records(m, d, precs, tpp, m->max_nlp);
        m->prec_bytes = fem::pair_rec_bytes(m->etype, m->per_elem_mat);
        m->n_pairs = tpp.back();
        if ((s = upload(m, &m->prec, precs.data(), precs.size(), st)) != FEM_OK) goto fail_out;
        if ((s = upload(m, &m->tile_pair_ptr, tpp.data(), tpp.size(), st)) != FEM_OK) goto fail_out;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            s = fail(FEM_ERR_CUDA, "cudaStreamSynchronize failed during upload");
            goto fail_out;
        }
    }
    {
        void* p = nullptr;
        const int aw = D == 2 ? 4 : 6;
        if ((s = zalloc(m, &p, (size_t)std::max<int64_t>(P.n_slots(), 1) * aw * 8, st)) != FEM_OK) goto fail_out;
        m->partial = p;
        if ((s = zalloc(m, &p, (size_t)P.n_tiles() * 4 * 8, st)) != FEM_OK) goto fail_out;
        m->tile_red = static_cast<double*>(p);
        if ((s = zalloc(m, &p, 16, st)) != FEM_OK) goto fail_out;
        m->tile_counter = static_cast<unsigned*>(p);
        if ((s = zalloc(m, &p, 16, st)) != FEM_OK) goto fail_out;
        m->status = static_cast<int*>(p);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        s = fail(FEM_ERR_CUDA, "cudaStreamSynchronize failed after upload");
        goto fail_out;
    }
    fill_info(P, &m->info);
    m->info.device_bytes = m->bytes;
    *out = m;
    return FEM_OK;
fail_out:
    free_all(m);
    delete m;
    return s;
}

fem_status fem_mesh_destroy(fem_mesh* m) {
    if (!m) return FEM_OK;
    cudaDeviceSynchronize();
    femi::solver_free(m);
    femi::lp_mesh_free(m);
    femi::sparse_free(m);
    femi::atomic_free(m);
    femi::ncm_free(m);
    free_all(m);
    delete m;
    return FEM_OK;
}

fem_status fem_mesh_set_moduli(fem_mesh* m, const double* mu, const double* lambda, void* stream) {
    if (!m || !mu || !lambda) return fail(FEM_ERR_ARG, "null mesh, mu or lambda");
    if (!m->per_elem_mat)
        return fail(FEM_ERR_ARG, "fem_mesh_set_moduli: the mesh was created with scalar moduli (no per-element slots)");
    const int64_t ne = m->info.n_elems;
    for (int64_t e = 0; e < ne; ++e)
        if (!(mu[e] > 0.0) || !std::isfinite(mu[e]) || !std::isfinite(lambda[e]))
            return fail(FEM_ERR_ARG, "fem_mesh_set_moduli: need finite mu > 0 and finite lambda");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const fem::Plan& P = m->plan;
    const int NG = m->etype == 0 ? 5 : (m->etype == 1 ? 10 : 0);
    const int64_t nr = P.n_rounds();
    // the (mu, lambda) pairs of every round, in record order (empty lanes 0),
    // copied into each round record's pair block by one strided copy per
    // precision
    for (int pi = 0; pi < 2; ++pi) {
        if (!m->rec[pi]) continue;
        const size_t ts = pi == 0 ? 8 : 4;
        std::vector<uint8_t> pairs((size_t)nr * 32 * 2 * ts, 0);
        for (int64_t r = 0; r < nr; ++r)
            for (int l = 0; l < 32; ++l) {
                const int32_t e = P.round_elem[r * 32 + l];
                if (e < 0) continue;
                uint8_t* dst = pairs.data() + ((size_t)r * 32 + l) * 2 * ts;
                if (pi == 0) {
                    const double v[2] = {mu[e], lambda[e]};
                    std::memcpy(dst, v, sizeof v);
                } else {
                    const float v[2] = {(float)mu[e], (float)lambda[e]};
                    std::memcpy(dst, v, sizeof v);
                }
            }
        const size_t off = (size_t)m->conn_bytes + ts * 32 * NG;
        CUDA_TRY(cudaMemcpy2DAsync(m->rec[pi] + off, (size_t)m->rec_bytes[pi], pairs.data(), 32 * 2 * ts, 32 * 2 * ts,
                                   (size_t)nr, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));  // `pairs` is a host temporary
    }
    if (m->prec && m->per_elem_mat) {
        // the (mu_A, mu_B, lam_A, lam_B) chunk of every pair record
        const int NCH = m->etype == 0 ? 3 : 5;
        const int64_t npr = (int64_t)(m->pair_elem.size() / 64);
        std::vector<float> chunk((size_t)npr * 128, 0.f);
        for (int64_t q = 0; q < npr; ++q)
            for (int l = 0; l < 32; ++l)
                for (int h = 0; h < 2; ++h) {
                    const int32_t e = m->pair_elem[(size_t)q * 64 + l * 2 + h];
                    if (e < 0) continue;
                    chunk[(size_t)q * 128 + l * 4 + h] = (float)mu[e];
                    chunk[(size_t)q * 128 + l * 4 + 2 + h] = (float)lambda[e];
                }
        CUDA_TRY(cudaMemcpy2DAsync(m->prec + 512 * (1 + NCH), (size_t)m->prec_bytes, chunk.data(), 512, 512,
                                   (size_t)npr, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    // host copies and what was derived from them: the ablation's element
    // arrays and the learned preconditioner's per-node statistics are rebuilt
    // on their next use
    m->mu_host.assign(mu, mu + ne);
    m->lam_host.assign(lambda, lambda + ne);
    femi::atomic_free(m);
    if (!m->conn_host.empty()) {
        const int64_t nn = m->info.n_nodes;
        std::vector<double> smu((size_t)nn, 0.0), slam((size_t)nn, 0.0), val((size_t)nn, 0.0);
        for (int64_t e = 0; e < ne; ++e)
            for (int a = 0; a < m->n_en; ++a) {
                const int32_t n = m->conn_host[e * m->n_en + a];
                smu[n] += mu[e];
                slam[n] += lambda[e];
                val[n] += 1.0;
            }
        for (int64_t n = 0; n < nn; ++n) {
            const double mb = val[n] > 0 ? smu[n] / val[n] : m->mu0;
            const double lb = val[n] > 0 ? slam[n] / val[n] : m->lam0;
            m->node_stats[n * 3 + 0] = (float)std::log(mb);
            m->node_stats[n * 3 + 1] = (float)std::log(lb / mb);
        }
        femi::lp_mesh_free(m);
    }
    return FEM_OK;
}

fem_status fem_mesh_get_info(const fem_mesh* m, fem_mesh_info* info) {
    if (!m || !info) return fail(FEM_ERR_ARG, "null argument");
    *info = m->info;
    return FEM_OK;
}

fem_status fem_energy(fem_mesh* m, int dtype, const void* u, double* out_dev, void* stream) {
    if (!u || !out_dev) return fail(FEM_ERR_ARG, "null u or output");
    return launch(m, dtype, fem::OP_ENERGY, u, nullptr, nullptr, out_dev, nullptr, nullptr, 0,
                  static_cast<cudaStream_t>(stream));
}

fem_status fem_energy_static(fem_mesh* m, int dtype, const void* u, double* out_dev, void* stream) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (!u || !out_dev) return fail(FEM_ERR_ARG, "null u or output");
    const int n_tiles = m->plan.n_tiles();
    if (n_tiles > FEM_STATIC_MAX_TILES)
        return fail(FEM_ERR_ARG, "fem_energy_static: the mesh has " + std::to_string(n_tiles) +
                                     " tiles but the static scratch holds " + std::to_string(FEM_STATIC_MAX_TILES) +
                                     "; use fem_energy or larger tiles");
    // every check of the call comes before the shared array is touched, so a
    // rejected call enqueues nothing (not even the counter's memset, which
    // would disturb another static call in flight)
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    if (dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    ReductionScratch scr{};
    fem_status s = static_scratch(&scr);
    if (s != FEM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero; the tile partials are written
    // before they are read
    CUDA_TRY(cudaMemsetAsync(scr.counter, 0, sizeof(unsigned), st));
    return launch(m, dtype, fem::OP_ENERGY, u, nullptr, nullptr, out_dev, nullptr, nullptr, 0, st, &scr);
}

fem_status fem_residual(fem_mesh* m, int dtype, const void* u, void* r, unsigned flags, void* stream) {
    if (!u || !r) return fail(FEM_ERR_ARG, "null u or r");
    if (u == r) return fail(FEM_ERR_ARG, "u and r must not alias");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    return launch(m, dtype, fem::OP_RESIDUAL, u, nullptr, r, nullptr, nullptr, nullptr, flags,
                  static_cast<cudaStream_t>(stream));
}

fem_status fem_hvp(fem_mesh* m, int dtype, const void* u, const void* v, void* y, unsigned flags,
                   double* vKv_dev, void* stream) {
    if (!u || !v || !y) return fail(FEM_ERR_ARG, "null u, v or y");
    if (y == u || y == v) return fail(FEM_ERR_ARG, "y must alias neither u nor v");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    return launch(m, dtype, fem::OP_HVP, u, v, y, vKv_dev, nullptr, nullptr, flags,
                  static_cast<cudaStream_t>(stream));
}

fem_status fem_block_diag(fem_mesh* m, int dtype, const void* u, void* D, void* stream) {
    if (!u || !D) return fail(FEM_ERR_ARG, "null u or D");
    return launch(m, dtype, fem::OP_BLOCKDIAG, u, nullptr, D, nullptr, nullptr, nullptr, 0,
                  static_cast<cudaStream_t>(stream));
}

fem_status fem_param_vjp(fem_mesh* m, int dtype, const void* u, const void* a, double* g_mu,
                         double* g_lam, void* stream) {
    if (!u || !a) return fail(FEM_ERR_ARG, "null u or a");
    return launch(m, dtype, fem::OP_PVJP, u, a, nullptr, nullptr, g_mu, g_lam, 0,
                  static_cast<cudaStream_t>(stream));
}

fem_status fem_sync_status(fem_mesh* m, void* stream, int32_t* flags) {
    if (!m || !flags) return fail(FEM_ERR_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *flags = h;
    return FEM_OK;
}

}  // extern "C"
