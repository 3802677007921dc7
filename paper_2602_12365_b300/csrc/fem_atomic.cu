// Ablation: the traditional element-centric scatter-add (Sec. 5, comparison
// with traditional assembly) on the same constitutive code.
//
// One thread per element in mesh order gathers its nodes' u (and v),
// evaluates P (residual) or dP (HVP) with the functions of fem_material.cuh,
// and adds its nodal forces into the global vector with floating-point
// atomicAdd.  Nothing orders the additions, so results agree with the tiled,
// coloured kernels to rounding but change in the last bits from run to run;
// the tiled kernels add every node's contributions in a fixed order.  Not on
// the method's path: the entry points exist to measure that difference.
// P1 elements (triangles, tetrahedra).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fem_b300.h"
#include "fem_internal.h"
#include "fem_kernels.cuh"

namespace femi {
struct AtomicData {
    int32_t* conn = nullptr;              // [ne][n_en], mesh order
    void* geo[2] = {nullptr, nullptr};    // [ne][D*D + 1] per precision (FP64, FP32)
    void* mod[2] = {nullptr, nullptr};    // [ne][2] (mu, lambda)
    std::vector<void*> allocs;
};

void atomic_free(fem_mesh* m) {
    if (!m || !m->atomic) return;
    for (void* p : m->atomic->allocs) cudaFree(p);
    delete m->atomic;
    m->atomic = nullptr;
}
}  // namespace femi

namespace {

constexpr int kT = 256;

fem_status fail(fem_status s, const std::string& msg) { return femi::set_error(s, msg); }

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(FEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define FEM_TRY(call)                \
    do {                             \
        fem_status s_ = (call);      \
        if (s_ != FEM_OK) return s_; \
    } while (0)

template <typename T>
fem_status upload(femi::AtomicData* A, T** dst, const std::vector<T>& src) {
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, std::max<size_t>(src.size(), 1) * sizeof(T)));
    A->allocs.push_back(p);
    CUDA_TRY(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = static_cast<T*>(p);
    return FEM_OK;
}

// element arrays in mesh order for precision pi (built on first use)
template <typename T>
fem_status prepare(fem_mesh* m, int pi) {
    if (!m->atomic) m->atomic = new femi::AtomicData();
    femi::AtomicData* A = m->atomic;
    if (A->geo[pi]) return FEM_OK;
    const int D = m->dim, NEN = m->n_en;
    const int64_t ne = m->info.n_elems;
    if ((int64_t)m->coords_host.size() != m->info.n_nodes * D || (int64_t)m->conn_host.size() != ne * NEN)
        return fail(FEM_ERR_ARG, "mesh geometry is not held");
    if (!A->conn) FEM_TRY(upload(A, &A->conn, m->conn_host));
    const int NG = D * D + 1;
    std::vector<T> geo((size_t)ne * NG), mod((size_t)ne * 2);
    double Xe[4 * 3], g[10];
    for (int64_t e = 0; e < ne; ++e) {
        for (int a = 0; a < NEN; ++a)
            for (int k = 0; k < D; ++k) Xe[a * D + k] = m->coords_host[(size_t)m->conn_host[e * NEN + a] * D + k];
        femi::p1_geometry(D, Xe, g);
        for (int j = 0; j < NG; ++j) geo[e * NG + j] = (T)g[j];
        mod[e * 2] = (T)(m->mu_host.empty() ? m->mu0 : m->mu_host[e]);
        mod[e * 2 + 1] = (T)(m->lam_host.empty() ? m->lam0 : m->lam_host[e]);
    }
    T *gp = nullptr, *mp = nullptr;
    FEM_TRY(upload(A, &gp, geo));
    FEM_TRY(upload(A, &mp, mod));
    A->geo[pi] = gp;
    A->mod[pi] = mp;
    return FEM_OK;
}

// one element per thread; the LAST vertex is the reference (its gradient is
// minus the sum of the others)
template <int D, typename T, int OP>
__global__ void __launch_bounds__(kT) atomic_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                    const T* __restrict__ geo, const T* __restrict__ mod,
                                                    const uint8_t* __restrict__ node_mask, const T* __restrict__ u,
                                                    const T* __restrict__ v, T* __restrict__ y, unsigned flags,
                                                    int* status) {
    constexpr int NEN = D + 1, NG = D * D + 1;
    for (int64_t e = blockIdx.x * (int64_t)kT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * kT) {
        int nd[NEN];
        uint8_t mk[NEN];
#pragma unroll
        for (int a = 0; a < NEN; ++a) {
            nd[a] = conn[e * NEN + a];
            mk[a] = node_mask[nd[a]];
        }
        T g[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) g[a][k] = geo[e * NG + a * D + k];
        const T wdJ = geo[e * NG + D * D];
        const T mu = mod[e * 2] * wdJ, lam = mod[e * 2 + 1] * wdJ;
        T ue[NEN][D], ve[NEN][D];
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                ue[a][c] = u[(int64_t)nd[a] * D + c];
                if constexpr (OP == fem::OP_HVP)
                    ve[a][c] = ((flags & FEM_MASK_IN) && ((mk[a] >> c) & 1)) ? T(0) : v[(int64_t)nd[a] * D + c];
            }
        T H[D][D], dF[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                T h = T(0), f = T(0);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    h = fma(ue[a][i] - ue[D][i], g[a][j], h);
                    if constexpr (OP == fem::OP_HVP) f = fma(ve[a][i] - ve[D][i], g[a][j], f);
                }
                H[i][j] = h;
                dF[i][j] = f;
            }
        fem::Kin<D, T> k;
        fem::kinematics<D, T>(H, k);
        if (!(k.ok & 1)) {
            atomicOr(status, FEM_FLAG_INVERTED);
            continue;  // an inverted element contributes nothing
        }
        T P[D][D];
        if constexpr (OP == fem::OP_RESIDUAL)
            fem::stress<D, T>(H, k, mu, lam, P);
        else
            fem::tangent<D, T>(dF, k, mu, lam, P);
        T fl[D];
#pragma unroll
        for (int c = 0; c < D; ++c) fl[c] = T(0);
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                T f;
                if (a < D) {
                    f = T(0);
#pragma unroll
                    for (int j = 0; j < D; ++j) f = fma(P[i][j], g[a][j], f);
                    fl[i] -= f;
                } else {
                    f = fl[i];
                }
                if ((flags & FEM_MASK_OUT) && ((mk[a] >> i) & 1)) continue;
                atomicAdd(y + (int64_t)nd[a] * D + i, f);
            }
    }
}

// Traditional assembly of K: the element stiffness column by column (the
// tangent on dF = e_j g_b^T for each vertex b and component j), each entry
// added with atomicAdd at its place in the CSR values.  Row (a, i) of the
// pattern holds D columns per node of N(a) in ascending order, so the entry
// (a i, b j) sits at row_ptr[a D + i] + D pos(b in N(a)) + j.
template <int D, typename T>
__global__ void __launch_bounds__(kT) assemble_kernel(int64_t ne, const int32_t* __restrict__ conn,
                                                      const T* __restrict__ geo, const T* __restrict__ mod,
                                                      const uint8_t* __restrict__ node_mask, const T* __restrict__ u,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const int64_t* __restrict__ node_ptr,
                                                      const int32_t* __restrict__ node_idx, T* __restrict__ vals,
                                                      unsigned flags, int* status) {
    constexpr int NEN = D + 1, NG = D * D + 1;
    for (int64_t e = blockIdx.x * (int64_t)kT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * kT) {
        int nd[NEN];
        uint8_t mk[NEN];
#pragma unroll
        for (int a = 0; a < NEN; ++a) {
            nd[a] = conn[e * NEN + a];
            mk[a] = node_mask[nd[a]];
        }
        T g[NEN][D];  // all vertices (the last: minus the sum of the others)
#pragma unroll
        for (int k = 0; k < D; ++k) g[D][k] = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                g[a][k] = geo[e * NG + a * D + k];
                g[D][k] -= g[a][k];
            }
        const T wdJ = geo[e * NG + D * D];
        const T mu = mod[e * 2] * wdJ, lam = mod[e * 2 + 1] * wdJ;
        T H[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                T h = T(0);
#pragma unroll
                for (int a = 0; a < D; ++a) h = fma(u[(int64_t)nd[a] * D + i] - u[(int64_t)nd[D] * D + i], g[a][j], h);
                H[i][j] = h;
            }
        fem::Kin<D, T> k;
        fem::kinematics<D, T>(H, k);
        if (!(k.ok & 1)) {
            atomicOr(status, FEM_FLAG_INVERTED);
            continue;
        }
        // where each vertex b sits in the node list of each vertex a
        int64_t base[NEN][NEN];
#pragma unroll
        for (int a = 0; a < NEN; ++a) {
            const int64_t q0 = node_ptr[nd[a]], q1 = node_ptr[nd[a] + 1];
            const int64_t r0 = row_ptr[(int64_t)nd[a] * D];
#pragma unroll
            for (int b = 0; b < NEN; ++b) {
                int64_t lo = q0, hi = q1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (node_idx[mid] < nd[b])
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                base[a][b] = r0 + (lo - q0) * D;
            }
        }
#pragma unroll
        for (int b = 0; b < NEN; ++b)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if ((flags & FEM_MASK_IN) && ((mk[b] >> j) & 1)) continue;
                T dF[D][D], dP[D][D];
#pragma unroll
                for (int r = 0; r < D; ++r)
#pragma unroll
                    for (int c = 0; c < D; ++c) dF[r][c] = (r == j) ? g[b][c] : T(0);
                fem::tangent<D, T>(dF, k, mu, lam, dP);
#pragma unroll
                for (int a = 0; a < NEN; ++a) {
                    const int64_t rowlen = (node_ptr[nd[a] + 1] - node_ptr[nd[a]]) * D;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        if ((flags & FEM_MASK_OUT) && ((mk[a] >> i) & 1)) continue;
                        T f = T(0);
#pragma unroll
                        for (int c = 0; c < D; ++c) f = fma(dP[i][c], g[a][c], f);
                        atomicAdd(vals + base[a][b] + i * rowlen + j, f);
                    }
                }
            }
    }
}

template <typename T>
fem_status run(fem_mesh* m, int op, const void* u, const void* v, void* y, unsigned flags, cudaStream_t st) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    FEM_TRY(prepare<T>(m, pi));
    const femi::AtomicData* A = m->atomic;
    const int64_t ne = m->info.n_elems;
    CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)m->info.n_nodes * m->dim * sizeof(T), st));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ne + kT - 1) / kT, 148 * 16));
    const T* gp = static_cast<const T*>(A->geo[pi]);
    const T* mp = static_cast<const T*>(A->mod[pi]);
    const T* uu = static_cast<const T*>(u);
    const T* vv = static_cast<const T*>(v);
    T* yy = static_cast<T*>(y);
    if (m->dim == 2) {
        if (op == fem::OP_RESIDUAL)
            atomic_kernel<2, T, fem::OP_RESIDUAL><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, uu, vv, yy,
                                                                     flags, m->status);
        else
            atomic_kernel<2, T, fem::OP_HVP><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, uu, vv, yy, flags,
                                                                m->status);
    } else {
        if (op == fem::OP_RESIDUAL)
            atomic_kernel<3, T, fem::OP_RESIDUAL><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, uu, vv, yy,
                                                                     flags, m->status);
        else
            atomic_kernel<3, T, fem::OP_HVP><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, uu, vv, yy, flags,
                                                                m->status);
    }
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
fem_status run_assemble(fem_mesh* m, const void* u, void* vals, unsigned flags, cudaStream_t st) {
    const int pi = sizeof(T) == 8 ? 0 : 1;
    FEM_TRY(prepare<T>(m, pi));
    const int64_t *row_ptr = nullptr, *node_ptr = nullptr;
    const int32_t* node_idx = nullptr;
    int64_t nnz = 0;
    FEM_TRY(femi::sparse_arrays(m, &row_ptr, &node_ptr, &node_idx, &nnz));
    const femi::AtomicData* A = m->atomic;
    const int64_t ne = m->info.n_elems;
    CUDA_TRY(cudaMemsetAsync(vals, 0, (size_t)nnz * sizeof(T), st));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ne + kT - 1) / kT, 148 * 16));
    const T* gp = static_cast<const T*>(A->geo[pi]);
    const T* mp = static_cast<const T*>(A->mod[pi]);
    if (m->dim == 2)
        assemble_kernel<2, T><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, static_cast<const T*>(u), row_ptr,
                                                   node_ptr, node_idx, static_cast<T*>(vals), flags, m->status);
    else
        assemble_kernel<3, T><<<grid, kT, 0, st>>>(ne, A->conn, gp, mp, m->node_mask, static_cast<const T*>(u), row_ptr,
                                                   node_ptr, node_idx, static_cast<T*>(vals), flags, m->status);
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

fem_status dispatch(fem_mesh* m, int dtype, int op, const void* u, const void* v, void* y, unsigned flags,
                    void* stream) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (m->etype == FEM_HEX8) return fail(FEM_ERR_ARG, "the atomic-scatter ablation covers P1 elements only");
    if (m->ncm) return fail(FEM_ERR_ARG, "the atomic-scatter ablation evaluates the Neo-Hookean law only");
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    if (dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return dtype == FEM_F64 ? run<double>(m, op, u, v, y, flags, st) : run<float>(m, op, u, v, y, flags, st);
}

}  // namespace

extern "C" {

fem_status fem_residual_atomic(fem_mesh* m, int dtype, const void* u, void* r, unsigned flags, void* stream) {
    if (!u || !r) return fail(FEM_ERR_ARG, "null u or r");
    if (u == r) return fail(FEM_ERR_ARG, "u and r must not alias");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    return dispatch(m, dtype, fem::OP_RESIDUAL, u, nullptr, r, flags, stream);
}

fem_status fem_hvp_atomic(fem_mesh* m, int dtype, const void* u, const void* v, void* y, unsigned flags,
                          void* stream) {
    if (!u || !v || !y) return fail(FEM_ERR_ARG, "null u, v or y");
    if (y == u || y == v) return fail(FEM_ERR_ARG, "y must alias neither u nor v");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    return dispatch(m, dtype, fem::OP_HVP, u, v, y, flags, stream);
}

fem_status fem_sparse_assemble_atomic(fem_mesh* m, int dtype, const void* u, unsigned flags, void* values,
                                      void* stream) {
    if (!u || !values) return fail(FEM_ERR_ARG, "null u or values");
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    if (m->etype == FEM_HEX8) return fail(FEM_ERR_ARG, "the atomic-scatter ablation covers P1 elements only");
    if (m->ncm) return fail(FEM_ERR_ARG, "the atomic-scatter ablation evaluates the Neo-Hookean law only");
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    if (dtype == FEM_F32 && m->precision != FEM_PREC_MIXED)
        return fail(FEM_ERR_ARG, "FEM_F32 needs a mesh created with FEM_PREC_MIXED");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return dtype == FEM_F64 ? run_assemble<double>(m, u, values, flags, st)
                            : run_assemble<float>(m, u, values, flags, st);
}

}  // extern "C"
