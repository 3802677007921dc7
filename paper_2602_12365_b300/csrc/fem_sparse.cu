// Sparse stiffness by colouring (Sec. 2.2, Algorithm 2; App. A and B).
//
// The DOF pattern of K (App. B) and a greedy distance-2 colouring of its
// columns (App. A) are built once per mesh on the host.  On the device,
// Algorithm 2 runs as one seeded HVP per colour: the seed e_c is 1 on the
// DOFs of colour c, the tile kernel's HVP gives K e_c, which is column c of
// the compressed Jacobian; since no two columns of one colour share a row,
// K_ij = Jcomp[colour(j)][i] for every pattern entry (i, j), and one gather
// pass writes the CSR values.  A CSR product y = K x closes the loop.
//
// Colouring on nodes: columns (n, a) and (m, b) share a row exactly when m
// lies within two element hops of n (N2(n) = union of N(p) over p in N(n),
// N(p) the nodes of p's elements, p included).  The column-order greedy on
// DOFs therefore takes, for node n in ascending order, the colours of every
// DOF of every earlier node of N2(n) as forbidden, and gives n's components
// a = 0, 1, .. the smallest free colours in turn: the same colouring as the
// DOF-level greedy, at node-level cost.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fem_b300.h"
#include "fem_internal.h"
#include "fem_kernels.cuh"

namespace femi {
struct SparseData {
    int64_t n_dofs = 0, nnz = 0;
    int32_t n_colors = 0;
    std::vector<int64_t> row_ptr;  // host CSR
    std::vector<int32_t> col_idx;
    std::vector<int32_t> colors;
    int64_t* d_row_ptr = nullptr;  // device copies
    int32_t* d_col_idx = nullptr;
    int32_t* d_colors = nullptr;
    int64_t* d_node_ptr = nullptr;  // N(n) as a node CSR (the pattern's block structure)
    int32_t* d_node_idx = nullptr;
    void* jcomp[2] = {nullptr, nullptr};  // [n_colors][n_dofs] per dtype (FP64, FP32)
    void* seeds[2] = {nullptr, nullptr};  // [n_colors][n_dofs]: e_c, built once per dtype
    std::vector<void*> allocs;
};

void sparse_free(fem_mesh* m) {
    if (!m || !m->sparse) return;
    for (void* p : m->sparse->allocs) cudaFree(p);
    delete m->sparse;
    m->sparse = nullptr;
}
}  // namespace femi

namespace {

constexpr int kT = 256;
constexpr int kMaxBlocks = 148 * 8;

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

int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kT - 1) / kT, kMaxBlocks));
}

template <typename T>
fem_status dalloc(femi::SparseData* d, T** p, size_t n) {
    void* q = nullptr;
    CUDA_TRY(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    d->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return FEM_OK;
}

// N(n): the nodes of n's elements (n included), ascending
void node_neighbours(int64_t nn, int64_t ne, int n_en, const int32_t* conn, std::vector<int64_t>& ptr,
                     std::vector<int32_t>& idx) {
    std::vector<int64_t> ep(nn + 1, 0);  // node -> elements
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < n_en; ++a) ep[conn[e * n_en + a] + 1]++;
    for (int64_t i = 0; i < nn; ++i) ep[i + 1] += ep[i];
    std::vector<int32_t> el(ep[nn]);
    std::vector<int64_t> fill(ep.begin(), ep.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < n_en; ++a) el[fill[conn[e * n_en + a]]++] = (int32_t)e;
    ptr.assign(nn + 1, 0);
    idx.clear();
    std::vector<int32_t> row;
    for (int64_t n = 0; n < nn; ++n) {
        row.clear();
        row.push_back((int32_t)n);
        for (int64_t q = ep[n]; q < ep[n + 1]; ++q)
            for (int a = 0; a < n_en; ++a) row.push_back(conn[(int64_t)el[q] * n_en + a]);
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        idx.insert(idx.end(), row.begin(), row.end());
        ptr[n + 1] = (int64_t)idx.size();
    }
}

// the DOF pattern and the colouring on the host
struct HostPattern {
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_idx, colors;
    int32_t n_colors = 0;
    std::vector<int64_t> node_ptr;  // N(n)
    std::vector<int32_t> node_idx;
};

fem_status host_pattern(int64_t nn, int64_t ne, int d, int n_en, const int32_t* conn, HostPattern& H) {
    if (nn * d > INT32_MAX) return fail(FEM_ERR_BADMESH, "sparse K: more than 2^31 - 1 DOFs");
    for (int64_t k = 0; k < ne * n_en; ++k)
        if (conn[k] < 0 || conn[k] >= nn) return fail(FEM_ERR_ARG, "connectivity entry out of range");
    std::vector<int64_t> np;
    std::vector<int32_t> ni;
    node_neighbours(nn, ne, n_en, conn, np, ni);
    const int64_t n_dofs = nn * d;
    // DOF pattern: row (n, a) holds (p, b) for p in N(n), b < d
    H.row_ptr.assign(n_dofs + 1, 0);
    int64_t nnz = 0;
    for (int64_t n = 0; n < nn; ++n)
        for (int a = 0; a < d; ++a) {
            nnz += (np[n + 1] - np[n]) * d;
            H.row_ptr[n * d + a + 1] = nnz;
        }
    H.col_idx.resize(nnz);
    for (int64_t n = 0; n < nn; ++n)
        for (int a = 0; a < d; ++a) {
            int64_t k = H.row_ptr[n * d + a];
            for (int64_t q = np[n]; q < np[n + 1]; ++q)
                for (int b = 0; b < d; ++b) H.col_idx[k++] = ni[q] * d + b;
        }
    // greedy distance-2 colouring, node by node (see the file comment)
    H.colors.assign(n_dofs, -1);
    std::vector<int64_t> stamp(64, -1);
    int32_t ncol = 0;
    for (int64_t n = 0; n < nn; ++n) {
        for (int64_t q = np[n]; q < np[n + 1]; ++q) {
            const int32_t p = ni[q];
            for (int64_t t = np[p]; t < np[p + 1]; ++t) {
                const int32_t mnode = ni[t];
                if (mnode >= n) continue;
                for (int b = 0; b < d; ++b) stamp[H.colors[(int64_t)mnode * d + b]] = n;
            }
        }
        for (int a = 0; a < d; ++a) {
            int32_t c = 0;
            while (c < (int32_t)stamp.size() && stamp[c] == n) ++c;
            if (c == (int32_t)stamp.size()) stamp.resize(stamp.size() * 2, -1);
            H.colors[n * d + a] = c;
            stamp[c] = n;  // taken for the node's next components
            ncol = std::max(ncol, c + 1);
        }
    }
    H.n_colors = ncol;
    H.node_ptr.swap(np);
    H.node_idx.swap(ni);
    return FEM_OK;
}

fem_status build_sparse_into(fem_mesh* m, femi::SparseData* S) {
    const int64_t nn = m->info.n_nodes, ne = m->info.n_elems;
    const int d = m->dim, n_en = m->n_en;
    if ((int64_t)m->conn_host.size() != ne * n_en) return fail(FEM_ERR_ARG, "mesh connectivity is not held");
    HostPattern H;
    FEM_TRY(host_pattern(nn, ne, d, n_en, m->conn_host.data(), H));
    S->n_dofs = nn * d;
    S->nnz = (int64_t)H.col_idx.size();
    S->n_colors = H.n_colors;
    S->row_ptr.swap(H.row_ptr);
    S->col_idx.swap(H.col_idx);
    S->colors.swap(H.colors);
    FEM_TRY(dalloc(S, &S->d_row_ptr, S->row_ptr.size()));
    FEM_TRY(dalloc(S, &S->d_col_idx, S->col_idx.size()));
    FEM_TRY(dalloc(S, &S->d_colors, S->colors.size()));
    FEM_TRY(dalloc(S, &S->d_node_ptr, H.node_ptr.size()));
    FEM_TRY(dalloc(S, &S->d_node_idx, H.node_idx.size()));
    CUDA_TRY(cudaMemcpy(S->d_node_ptr, H.node_ptr.data(), H.node_ptr.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(S->d_node_idx, H.node_idx.data(), H.node_idx.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(S->d_row_ptr, S->row_ptr.data(), S->row_ptr.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(S->d_col_idx, S->col_idx.data(), S->col_idx.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(S->d_colors, S->colors.data(), S->colors.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
    return FEM_OK;
}

// pattern and colouring on first use; the mesh keeps them only when complete
fem_status build_sparse(fem_mesh* m) {
    if (m->sparse) return FEM_OK;
    auto* S = new femi::SparseData();
    const fem_status s = build_sparse_into(m, S);
    if (s != FEM_OK) {
        for (void* p : S->allocs) cudaFree(p);
        delete S;
        return s;
    }
    m->sparse = S;
    return FEM_OK;
}

// the seeds of all colours: e_c[j] = 1 on the DOFs j of colour c ([n_colors][n])
template <typename T>
__global__ void __launch_bounds__(kT) seed_kernel(int64_t n, int32_t n_colors, const int32_t* __restrict__ colors,
                                                  T* __restrict__ e) {
    const int64_t total = n * n_colors;
    for (int64_t k = blockIdx.x * (int64_t)kT + threadIdx.x; k < total; k += (int64_t)gridDim.x * kT) {
        const int64_t c = k / n, j = k - c * n;
        e[k] = colors[j] == (int32_t)c ? T(1) : T(0);
    }
}

// Algorithm 2's decompression: K_ij = Jcomp[colour(j)][i], a warp per row
template <typename T>
__global__ void __launch_bounds__(kT) decompress_kernel(int64_t n_rows, const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col_idx,
                                                        const int32_t* __restrict__ colors,
                                                        const T* __restrict__ jcomp, T* __restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kT / 32);
    for (int64_t i = blockIdx.x * (int64_t)(kT / 32) + (threadIdx.x >> 5); i < n_rows; i += warps) {
        const int64_t k0 = row_ptr[i], k1 = row_ptr[i + 1];
        for (int64_t k = k0 + lane; k < k1; k += 32) vals[k] = jcomp[(int64_t)colors[col_idx[k]] * n_rows + i];
    }
}

int pix(int dtype) { return dtype == FEM_F64 ? 0 : 1; }

}  // namespace

namespace femi {
fem_status sparse_arrays(fem_mesh* m, const int64_t** row_ptr, const int64_t** node_ptr, const int32_t** node_idx,
                         int64_t* nnz) {
    FEM_TRY(build_sparse(m));
    *row_ptr = m->sparse->d_row_ptr;
    *node_ptr = m->sparse->d_node_ptr;
    *node_idx = m->sparse->d_node_idx;
    *nnz = m->sparse->nnz;
    return FEM_OK;
}
}  // namespace femi

extern "C" {

fem_status fem_sparse_info(fem_mesh* m, int64_t* nnz, int32_t* n_colors) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    FEM_TRY(build_sparse(m));
    if (nnz) *nnz = m->sparse->nnz;
    if (n_colors) *n_colors = m->sparse->n_colors;
    return FEM_OK;
}

fem_status fem_sparse_pattern_desc(const fem_mesh_desc* desc, int64_t* nnz, int32_t* n_colors, int64_t* row_ptr,
                                   int32_t* col_idx, int32_t* colors) {
    if (!desc || !desc->conn) return fail(FEM_ERR_ARG, "null descriptor or connectivity");
    if (desc->elem_type < 0 || desc->elem_type > 2) return fail(FEM_ERR_ARG, "elem_type must be 0, 1 or 2");
    if (desc->n_nodes <= 0 || desc->n_elems <= 0) return fail(FEM_ERR_ARG, "empty mesh");
    const int d = desc->elem_type == FEM_TRI3 ? 2 : 3;
    const int n_en = desc->elem_type == FEM_TRI3 ? 3 : (desc->elem_type == FEM_TET4 ? 4 : 8);
    HostPattern H;
    FEM_TRY(host_pattern(desc->n_nodes, desc->n_elems, d, n_en, desc->conn, H));
    if (nnz) *nnz = (int64_t)H.col_idx.size();
    if (n_colors) *n_colors = H.n_colors;
    if (row_ptr) std::copy(H.row_ptr.begin(), H.row_ptr.end(), row_ptr);
    if (col_idx) std::copy(H.col_idx.begin(), H.col_idx.end(), col_idx);
    if (colors) std::copy(H.colors.begin(), H.colors.end(), colors);
    return FEM_OK;
}

fem_status fem_sparse_pattern(fem_mesh* m, int64_t* row_ptr, int32_t* col_idx, int32_t* colors) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    FEM_TRY(build_sparse(m));
    const femi::SparseData* S = m->sparse;
    if (row_ptr) std::copy(S->row_ptr.begin(), S->row_ptr.end(), row_ptr);
    if (col_idx) std::copy(S->col_idx.begin(), S->col_idx.end(), col_idx);
    if (colors) std::copy(S->colors.begin(), S->colors.end(), colors);
    return FEM_OK;
}

fem_status fem_sparse_assemble(fem_mesh* m, int dtype, const void* u, unsigned flags, void* values, void* stream) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (!u || !values) return fail(FEM_ERR_ARG, "null u or values");
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    if (flags & ~(unsigned)FEM_MASK_BOTH) return fail(FEM_ERR_ARG, "flags: only FEM_MASK_IN and FEM_MASK_OUT");
    FEM_TRY(build_sparse(m));
    femi::SparseData* S = m->sparse;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int pi = pix(dtype);
    const size_t es = dtype == FEM_F64 ? sizeof(double) : sizeof(float);
    if (!S->jcomp[pi]) {  // workspace and the seeds of all colours, once per dtype
        unsigned char *jc = nullptr, *sd = nullptr;
        FEM_TRY(dalloc(S, &jc, (size_t)S->n_colors * S->n_dofs * es));
        FEM_TRY(dalloc(S, &sd, (size_t)S->n_colors * S->n_dofs * es));
        const int gs = grid_for(S->n_dofs * S->n_colors);
        if (dtype == FEM_F64)
            seed_kernel<double><<<gs, kT, 0, st>>>(S->n_dofs, S->n_colors, S->d_colors, reinterpret_cast<double*>(sd));
        else
            seed_kernel<float><<<gs, kT, 0, st>>>(S->n_dofs, S->n_colors, S->d_colors, reinterpret_cast<float*>(sd));
        CUDA_TRY(cudaGetLastError());
        S->jcomp[pi] = jc;
        S->seeds[pi] = sd;
    }
    // one state for all colours: Neo-Hookean meshes store the linearisation
    // once and every seeded HVP reads it; with a neural constitutive model
    // the first HVP evaluates the network at u and the others reuse it
    const bool lin = !m->ncm;
    if (lin) FEM_TRY(femi::run_op(m, dtype, fem::OP_LINEARIZE, u, nullptr, nullptr, nullptr, 0, st, nullptr));
    for (int32_t c = 0; c < S->n_colors; ++c) {
        void* col = static_cast<unsigned char*>(S->jcomp[pi]) + (size_t)c * S->n_dofs * es;
        const void* seed = static_cast<const unsigned char*>(S->seeds[pi]) + (size_t)c * S->n_dofs * es;
        const unsigned fixed = lin ? femi::kFlagUseLin : (c > 0 ? femi::kFlagNcmCurrent : 0u);
        FEM_TRY(femi::run_op(m, dtype, fem::OP_HVP, u, seed, col, nullptr, flags | fixed, st, nullptr));
    }
    const int gd = grid_for(S->n_dofs * 32);
    if (dtype == FEM_F64)
        decompress_kernel<double><<<gd, kT, 0, st>>>(S->n_dofs, S->d_row_ptr, S->d_col_idx, S->d_colors,
                                                     static_cast<const double*>(S->jcomp[pi]),
                                                     static_cast<double*>(values));
    else
        decompress_kernel<float><<<gd, kT, 0, st>>>(S->n_dofs, S->d_row_ptr, S->d_col_idx, S->d_colors,
                                                    static_cast<const float*>(S->jcomp[pi]),
                                                    static_cast<float*>(values));
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}


}  // extern "C"
