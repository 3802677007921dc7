// The CSR product y = K x of the sparse-K route (Sec. 2.2, Algorithm 2):
// the matrix that fem_sparse_assemble fills, applied with the pattern's
// node-block structure (fem_sparse.cu builds the pattern and its device
// copies; this file holds only the product, so that its measurements are
// tied to this kernel alone).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "fem_b300.h"
#include "fem_internal.h"

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

// y = K x on the CSR values, read through the pattern's block structure:
// the D rows of node n hold the same columns, D per node p of N(n) in order,
// so row (n, r) has value q D + b at column p D + b for the q-th node p of
// N(n).  A half-warp takes node n; each lane sums a strided part of the
// (q, b) entries for all D rows (one node id per entry instead of a column
// index per value, and consecutive lanes on consecutive values), then a
// fixed butterfly adds the parts.  (Measured on the 64^3 tet mesh: this
// mapping beats a lane per D x D block and unrolled or register-capped
// variants.)
template <int D, typename T>
__global__ void __launch_bounds__(kT) spmv_kernel(int64_t nn, const int64_t* __restrict__ row_ptr,
                                                  const int64_t* __restrict__ node_ptr,
                                                  const int32_t* __restrict__ node_idx, const T* __restrict__ vals,
                                                  const T* __restrict__ x, T* __restrict__ y) {
    constexpr int L = 16;
    const int lane = threadIdx.x & 31, half = lane / L, sub = lane & (L - 1);
    const int64_t warps = (int64_t)gridDim.x * (kT / 32);
    // the loop bound is the same for all lanes of a warp (the shuffles need them all)
    for (int64_t w = blockIdx.x * (int64_t)(kT / 32) + (threadIdx.x >> 5); 2 * w < nn; w += warps) {
        const int64_t n = 2 * w + half;
        T s[D];
#pragma unroll
        for (int r = 0; r < D; ++r) s[r] = T(0);
        if (n < nn) {
            const int64_t q0 = node_ptr[n];
            const int len = (int)(node_ptr[n + 1] - q0) * D;  // entries per row
            const T* v0 = vals + row_ptr[n * D];
            for (int e = sub; e < len; e += L) {
                const int q = e / D, b = e - q * D;
                const T xv = x[(int64_t)node_idx[q0 + q] * D + b];
#pragma unroll
                for (int r = 0; r < D; ++r) s[r] += v0[(int64_t)r * len + e] * xv;
            }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
            for (int r = 0; r < D; ++r) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o, L);
        if (n < nn && sub < D) {
            T t = s[0];
#pragma unroll
            for (int r = 1; r < D; ++r)
                if (sub == r) t = s[r];
            y[n * D + sub] = t;
        }
    }
}

}  // namespace

extern "C" {

fem_status fem_sparse_spmv(fem_mesh* m, int dtype, const void* values, const void* x, void* y, void* stream) {
    if (!m) return fail(FEM_ERR_ARG, "null mesh");
    if (!values || !x || !y) return fail(FEM_ERR_ARG, "null values, x or y");
    if (x == y) return fail(FEM_ERR_ARG, "x and y must not alias");
    if (dtype != FEM_F64 && dtype != FEM_F32) return fail(FEM_ERR_ARG, "dtype must be FEM_F64 or FEM_F32");
    const int64_t *row_ptr = nullptr, *node_ptr = nullptr;
    const int32_t* node_idx = nullptr;
    int64_t nnz = 0;
    FEM_TRY(femi::sparse_arrays(m, &row_ptr, &node_ptr, &node_idx, &nnz));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nn = m->info.n_nodes;
    const int g = grid_for(nn * 16);
    if (m->dim == 2) {
        if (dtype == FEM_F64)
            spmv_kernel<2, double><<<g, kT, 0, st>>>(nn, row_ptr, node_ptr, node_idx,
                                                     static_cast<const double*>(values), static_cast<const double*>(x),
                                                     static_cast<double*>(y));
        else
            spmv_kernel<2, float><<<g, kT, 0, st>>>(nn, row_ptr, node_ptr, node_idx,
                                                    static_cast<const float*>(values), static_cast<const float*>(x),
                                                    static_cast<float*>(y));
    } else {
        if (dtype == FEM_F64)
            spmv_kernel<3, double><<<g, kT, 0, st>>>(nn, row_ptr, node_ptr, node_idx,
                                                     static_cast<const double*>(values), static_cast<const double*>(x),
                                                     static_cast<double*>(y));
        else
            spmv_kernel<3, float><<<g, kT, 0, st>>>(nn, row_ptr, node_ptr, node_idx,
                                                    static_cast<const float*>(values), static_cast<const float*>(x),
                                                    static_cast<float*>(y));
    }
    CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // extern "C"
