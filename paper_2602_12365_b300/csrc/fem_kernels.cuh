// Tile kernels of the energy-based FEM hot path (sm_103a).
//
// Per element (Algorithm 1 of arXiv 2602.12365): gather the nodal values,
// form H = grad u = sum_a u_a (x) grad N_a and F = I + H, evaluate the
// Neo-Hookean density / stress / tangent action (fem_material.cuh), multiply
// by w_q det J and scatter.  P1 elements read precomputed grad N_a and
// w det J from their round record; Q1 hexahedra rebuild J from the staged
// nodal coordinates at each of the 2x2x2 Gauss points.
//
// Work decomposition (fem_plan.h): one CTA of kWarps warps owns one tile.
//   prologue  bulk copies (TMA engine) of the first round records of every
//             warp start; the tile's nodal u (v, X), node ids and partial
//             slots are gathered into shared memory; accumulators zeroed.
//   rounds    warp w runs a contiguous range of the tile's rounds, one
//             element per lane (two elements per lane, packed in FP32x2
//             pairs, for FP32 P1 calls), and accumulates into its own
//             shared-memory copy.  The elements of one round share no node,
//             so lanes never collide; rounds of one warp are applied in
//             order.  Records stream through a per-warp ring of kStages
//             stages filled by cp.async.bulk and guarded by mbarriers (every
//             wait is bounded and reports FEM_FLAG_TIMEOUT).
//   epilogue  the warp copies are summed in warp order; nodes private to the
//             tile are written, nodes shared with other tiles go to their
//             fixed partial slot.
// finalize_kernel (launched with programmatic dependent launch) sums each
// shared node's slots in slot (= tile) order.  Every sum has a fixed order,
// so results are bitwise reproducible and no floating-point atomic is used.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fem_material.cuh"
#include "fem_vec.cuh"

namespace fem {

// Tile shape (compile-time tuning knobs; the defaults are the measured best)
#ifndef FEM_TILE_WARPS
#define FEM_TILE_WARPS 4
#endif
#ifndef FEM_RING_STAGES
#define FEM_RING_STAGES 1
#endif
#ifndef FEM_PAIR_FP32
#define FEM_PAIR_FP32 0
#endif
#ifndef FEM_DUAL_ROUNDS
#define FEM_DUAL_ROUNDS 1
#endif
#ifndef FEM_DUAL_LIN
#define FEM_DUAL_LIN 0  // two rounds per iteration for the stored-linearisation HVP (measured slower)
#endif
constexpr int kWarps = FEM_TILE_WARPS;   // warps per tile (one accumulator copy each)
constexpr int kThreads = 32 * kWarps;
constexpr int kStages = FEM_RING_STAGES;  // ring stages per warp
constexpr int kSpinLimit = 1 << 20;  // bounded mbarrier waits
constexpr int kFinThreads = 256;

// OP_NCM_INV writes each P1 element's (I1 - 3, J - 1) in record order: the
// inputs of the neural constitutive model's network (coefficient pass)
// OP_LINEARIZE writes each P1 element's linearisation at u (F^-T, w mu,
// w (mu - lambda ln J), w lambda: 12 values, record order) for HVPs at the
// same state (the PCG of a Newton step), which then skip u, F and its
// inverse and logarithm (tile_kernel<..., LIN>)
enum Op { OP_ENERGY = 0, OP_RESIDUAL = 1, OP_HVP = 2, OP_BLOCKDIAG = 3, OP_PVJP = 4, OP_NCM_INV = 5, OP_LINEARIZE = 6 };
constexpr int kLinVals = 12;  // per element: F^-T (9), w mu, w (mu - lambda ln J), w lambda
// Q1: per Gauss point A = F^-T J^-T (9), C = J^-1 J^-T (6: 00 11 22 01 02 12),
// det J mu, det J (mu - lambda ln J), det J lambda, 2 zeros (J = dx/dxi);
// stored lane-major in 16-byte chunks: chunk c of point q of lane l in
// round r at ((r * 8 + q) * NCH + c) * 32 + l, NCH = kHexLinVals * size / 16
constexpr int kHexLinVals = 20;
template <typename T>
__host__ __device__ constexpr int hex_lin_chunks() {
    return kHexLinVals * (int)sizeof(T) / 16;
}
// Gauss points of the Q1 linearisation in flight per lane (a per-warp
// shared-memory ring of [stage][chunk][lane] 16-byte chunks, filled by
// cp.async kHexLinStages - 1 points ahead of their use)
__host__ __device__ constexpr int hex_lin_stages(int tsize) { return tsize == 4 ? 3 : 2; }

template <int ET>
struct ElemT;
template <>
struct ElemT<0> {  // P1 triangle, plane strain, 1 point
    static constexpr int D = 2, NEN = 3, PAD = 4, NG = 5, VW = 2;
};
template <>
struct ElemT<1> {  // P1 tetrahedron, 1 point
    static constexpr int D = 3, NEN = 4, PAD = 4, NG = 10, VW = 4;
};
template <>
struct ElemT<2> {  // Q1 hexahedron, 2x2x2 Gauss
    static constexpr int D = 3, NEN = 8, PAD = 8, NG = 0, VW = 4;
};

// rounds per warp iteration: FEM_PAIR_FP32 packs two FP32 P1 rounds into
// FP32x2 pairs; FEM_DUAL_ROUNDS gives each lane two independent elements (one
// per round) computed with scalar arithmetic, so that their dependency chains
// interleave, and fetches the two round records in one copy (FP32 P1 energy
// and residual; with FEM_DUAL_LIN also the HVP from a stored linearisation,
// which fits but measured slower; the full HVP's larger node buffers leave no
// room for the second record in shared memory without losing a resident CTA)
__host__ __device__ constexpr int rounds_per_iter(int et, int tsize, int op, bool lin = false) {
    return (et != 2 && tsize == 4 &&
            (FEM_PAIR_FP32 || (FEM_DUAL_ROUNDS && (op == OP_ENERGY || op == OP_RESIDUAL)) ||
             (FEM_DUAL_LIN && lin && op == OP_HVP)))
               ? 2
               : 1;
}

// ---------------------------------------------------------------------------
// shared-memory layout (bytes), identical on host and device.  Two node
// buffers (the current tile's and the next tile's: nodal u, v, X, node ids,
// partial slots, Dirichlet bits), the per-warp accumulator copies, reduction
// scratch, the CTA's tile table, the per-warp record ring and the mbarriers.
// ---------------------------------------------------------------------------
constexpr int kMaxTilesPerCta = 16;
// Q1 tiles are a quarter of the P1 ones (their node buffers are larger) and
// their kernels hold two CTAs per SM: a cap of 32 keeps the grid at one CTA
// per resident slot on the 128^3 mesh (8192 tiles) instead of a second,
// partial wave.
__host__ __device__ constexpr int max_tiles_per_cta(int et) { return et == 2 ? 2 * kMaxTilesPerCta : kMaxTilesPerCta; }

struct SmemLayout {
    int off_u, off_v, off_x, buf_bytes;  // inside one node buffer
    int off_buf0, off_buf1, off_acc, acc_bytes, off_red, off_tab, off_ring, off_lin, off_bar, total, aw,
        stage_bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int align128(int x) { return (x + 127) & ~127; }

// nlp: the largest padded tile node count
// lin: the HVP from a stored linearisation (no u buffer; each ring stage
// also carries the rounds' 32 x kLinVals values)
__host__ __device__ inline SmemLayout smem_layout(int et, int tsize, int op, int nlp, int rec_bytes, bool lin = false) {
    SmemLayout L;
    const int D = et == 0 ? 2 : 3;
    const int VW = D == 2 ? 2 : 4;
    const int vec = VW * tsize;
    L.aw = (op == OP_BLOCKDIAG) ? (D == 2 ? 4 : 6) : VW;
    const bool need_v = (op == OP_HVP || op == OP_PVJP);
    const bool need_acc = (op == OP_RESIDUAL || op == OP_HVP || op == OP_BLOCKDIAG);
    int o = 0;
    L.off_u = o;
    if (!lin) o = align16(o + nlp * vec);
    L.off_v = o;
    if (need_v) o = align16(o + nlp * vec);
    L.off_x = o;
    if (et == 2 && !lin) o = align16(o + nlp * vec);
    L.buf_bytes = align128(o);
    L.off_buf0 = 0;
    L.off_buf1 = L.buf_bytes;
    o = 2 * L.buf_bytes;
    L.off_acc = o;
    L.acc_bytes = need_acc ? align16(kWarps * nlp * L.aw * tsize) : 0;
    o += L.acc_bytes;
    L.off_red = o;
    o = align16(o + kWarps * 4 * 8 + 16);
    L.off_tab = o;
    o = align16(o + max_tiles_per_cta(et) * 16);
    // (Q1 reads its per-point linearisation from global memory, not the ring)
    L.stage_bytes = rounds_per_iter(et, tsize, op, lin) * (rec_bytes + (lin && et != 2 ? 32 * kLinVals * tsize : 0));
    L.off_ring = o = align128(o);
    o += kWarps * kStages * L.stage_bytes;
    L.off_lin = o = align16(o);
    if (et == 2 && lin) o += kWarps * hex_lin_stages(tsize) * 32 * kHexLinVals * tsize;
    L.off_bar = o = align16(o);
    o += kWarps * kStages * 8;
    L.total = align16(o);
    return L;
}

struct KParams {
    // plan
    const int32_t* tile_round_ptr;
    const int64_t* tile_node_ptr;
    const int32_t* node_gid;
    const int32_t* node_slot;
    const uint8_t* round_nvalid;
    const int32_t* round_elem;
    // round records: u16 conn[32][PAD] | T elem[32][stride] (elem: grad N_0..
    // grad N_{NEN-2}, w det J for P1; then mu, lambda when has_mat)
    const uint8_t* rec;
    int rec_bytes;
    int conn_bytes;
    int stride;
    int has_mat;
    const int32_t* slot_owner;
    const int4* shared_info;  // [n_shared] first slot, end slot, node, Dirichlet bits
    int n_shared;
    const int32_t* orphans;
    int n_orphans;
    const uint8_t* node_mask;        // [n_nodes] Dirichlet bits
    const uint8_t* node_mask_local;  // [n_local] Dirichlet bits per tile-local node
    const void* X;  // Q1: nodal coordinates [n_nodes][3] in the kernel's dtype
    int n_tiles;
    int max_nlp;  // largest padded tile node count
    double mu0, lam0;
    // workspace
    void* partial;
    double* tile_red;
    unsigned* tile_counter;
    int* status;
    const int* skip;  // device flag: the call does nothing when *skip != 0 (may be null)
    int vkv_tiles;    // HVP: write the per-tile vKv partials (tile_red) even without out_scalar
    // neural constitutive model, in record order (round * 32 + lane): the
    // network's coefficients [8] per element (NCM kernels) and the invariants
    // [2] per element (OP_NCM_INV)
    const void* ncm_coef;
    void* ncm_inv;
    // linearisation [n_rounds * 32][kLinVals] in record order (OP_LINEARIZE
    // writes it, the LIN HVP streams it through the record ring)
    void* lin;
    // pair records of the FP32 P1 pair kernels (fem_pair.cuh): two rounds
    // per lane and record, tile by tile and warp by warp
    const uint8_t* prec;
    int prec_bytes;
    const int32_t* tile_pair_ptr;
    // call
    const void* u;
    const void* v;
    void* out;
    double* out_scalar;
    double* out_mu;
    double* out_lam;
    unsigned flags;
};

// ---------------------------------------------------------------------------
// bulk copies (TMA engine), mbarriers and dependent launch, by inline PTX
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// arm the barrier for `bytes` and start one bulk copy global -> shared
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// two bulk copies completing one mbarrier phase
__device__ __forceinline__ void bulk_load2(void* dst0, const void* src0, uint32_t b0, void* dst1, const void* src1,
                                           uint32_t b1, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(b0 + b1)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst0)),
        "l"(src0), "r"(b0), "r"(smem_u32(bar))
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst1)),
        "l"(src1), "r"(b1), "r"(smem_u32(bar))
        : "memory");
}

// L2 policy for data read once per call (the P1 stored linearisation and its
// round records in the PCG, 150 MB on tet64): evicted first, so that the
// solver's vectors (45 MB on tet64), reused every iteration, stay in L2.  (Q1
// meshes of the benchmark's size have vectors larger than L2 and do not use it.)
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_load2 with an L2 cache policy on both copies
__device__ __forceinline__ void bulk_load2_hint(void* dst0, const void* src0, uint32_t b0, void* dst1,
                                                const void* src1, uint32_t b1, uint64_t* bar, uint64_t pol) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(b0 + b1)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst0)),
        "l"(src0), "r"(b0), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst1)),
        "l"(src1), "r"(b1), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false if the copy did not land within the limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// expect `bytes` on the barrier and arrive once (one per phase)
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// bulk copy that completes bytes on `bar` without arriving
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// asynchronous 4- or 8-byte global -> shared copies (completion by group)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// 16-byte global -> shared copy through L2 only
__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// shared-memory vectors
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }

template <int VW, typename T>
__device__ __forceinline__ void lds_vec(const T* base, int i, T* out) {
    if constexpr (VW == 4 && sizeof(T) == 4) {
        float4 t = reinterpret_cast<const float4*>(base)[i];
        out[0] = t.x;
        out[1] = t.y;
        out[2] = t.z;
        out[3] = t.w;
    } else if constexpr (VW == 2 && sizeof(T) == 4) {
        float2 t = reinterpret_cast<const float2*>(base)[i];
        out[0] = t.x;
        out[1] = t.y;
    } else if constexpr (VW == 4) {
        double2 a = reinterpret_cast<const double2*>(base)[2 * i];
        double2 b = reinterpret_cast<const double2*>(base)[2 * i + 1];
        out[0] = a.x;
        out[1] = a.y;
        out[2] = b.x;
        out[3] = b.y;
    } else {
        double2 a = reinterpret_cast<const double2*>(base)[i];
        out[0] = a.x;
        out[1] = a.y;
    }
}

template <int VW, typename T>
__device__ __forceinline__ void sts_vec(T* base, int i, const T* in) {
    if constexpr (VW == 4 && sizeof(T) == 4) {
        reinterpret_cast<float4*>(base)[i] = make_float4(in[0], in[1], in[2], in[3]);
    } else if constexpr (VW == 2 && sizeof(T) == 4) {
        reinterpret_cast<float2*>(base)[i] = make_float2(in[0], in[1]);
    } else if constexpr (VW == 4) {
        reinterpret_cast<double2*>(base)[2 * i] = make_double2(in[0], in[1]);
        reinterpret_cast<double2*>(base)[2 * i + 1] = make_double2(in[2], in[3]);
    } else {
        reinterpret_cast<double2*>(base)[i] = make_double2(in[0], in[1]);
    }
}

// Lane's geometry from a round record in shared memory.  The N geometry
// scalars of the round's 32 elements are stored in 16-byte chunks: chunk k
// holds scalars [k CW, k CW + w) of every lane, lane-major (CW = 4 floats or
// 2 doubles; w = CW except for the last chunk), so each chunk is one
// conflict-free vector load per lane.
template <typename T, int N>
__device__ __forceinline__ void lds_chunks(const T* el0, int lane, T (&dst)[N]) {
    constexpr int CW = 16 / (int)sizeof(T);
    static_assert(N % CW != 3, "a 3-wide chunk has no vector load");
#pragma unroll
    for (int k = 0; k * CW < N; ++k) {
        const int w = (N - k * CW < CW) ? N - k * CW : CW;
        const T* src = el0 + 32 * k * CW;
        if constexpr (sizeof(T) == 4) {
            if (w == 4) {
                const float4 t = reinterpret_cast<const float4*>(src)[lane];
                dst[4 * k + 0] = t.x;
                dst[4 * k + 1] = t.y;
                dst[4 * k + 2] = t.z;
                dst[4 * k + 3] = t.w;
            } else if (w == 2) {
                const float2 t = reinterpret_cast<const float2*>(src)[lane];
                dst[4 * k + 0] = t.x;
                dst[4 * k + 1] = t.y;
            } else {
                dst[4 * k] = src[lane];
            }
        } else {
            if (w == 2) {
                const double2 t = reinterpret_cast<const double2*>(src)[lane];
                dst[2 * k + 0] = t.x;
                dst[2 * k + 1] = t.y;
            } else {
                dst[2 * k] = src[lane];
            }
        }
    }
}

// one half of a lane's work: an element of a round record
template <int ET, typename T>
struct Half {
    static constexpr int NEN = ElemT<ET>::NEN, NG = ElemT<ET>::NG;
    int cn[NEN];
    T ed[NG + 2];  // geometry, mu, lambda
};

// Read lane's element of a round record (if the record is there and the lane
// is not empty); returns whether it holds an element.  Empty lanes get node 0
// and zero geometry so they compute harmlessly.
template <int ET, typename T>
__device__ __forceinline__ bool read_half(const uint8_t* rec, int lane, bool present, const KParams& p,
                                          T mu0, T lam0, Half<ET, T>& h) {
    using E = ElemT<ET>;
    bool valid = false;
    if (present) {
        if constexpr (E::PAD == 4) {
            const uint2 w = reinterpret_cast<const uint2*>(rec)[lane];
            h.cn[0] = w.x & 0xffff;
            h.cn[1] = w.x >> 16;
            h.cn[2] = w.y & 0xffff;
            if constexpr (E::NEN == 4) h.cn[3] = w.y >> 16;
        } else {
            const uint4 w = reinterpret_cast<const uint4*>(rec)[lane];
            h.cn[0] = w.x & 0xffff;
            h.cn[1] = w.x >> 16;
            h.cn[2] = w.y & 0xffff;
            h.cn[3] = w.y >> 16;
            h.cn[4] = w.z & 0xffff;
            h.cn[5] = w.z >> 16;
            h.cn[6] = w.w & 0xffff;
            h.cn[7] = w.w >> 16;
        }
        valid = h.cn[0] != 0xFFFF;
    }
    if (!valid) {
#pragma unroll
        for (int a = 0; a < E::NEN; ++a) h.cn[a] = 0;
#pragma unroll
        for (int j = 0; j < E::NG + 2; ++j) h.ed[j] = T(0);
        return false;
    }
    const T* el0 = reinterpret_cast<const T*>(rec + p.conn_bytes);
    if constexpr (E::NG > 0) {
        T g[E::NG];
        lds_chunks<T, E::NG>(el0, lane, g);
#pragma unroll
        for (int j = 0; j < E::NG; ++j) h.ed[j] = g[j];
    }
    if (p.has_mat) {  // (mu, lambda) pairs after the geometry chunks
        using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        const T2 m = reinterpret_cast<const T2*>(el0 + 32 * E::NG)[lane];
        h.ed[E::NG] = m.x;
        h.ed[E::NG + 1] = m.y;
    } else {
        h.ed[E::NG] = mu0;
        h.ed[E::NG + 1] = lam0;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Q1 reference gradients at the 2x2x2 Gauss points (compile-time constants)
// ---------------------------------------------------------------------------
constexpr double kGauss = 0.57735026918962576451;  // 1/sqrt(3)

__host__ __device__ constexpr int hex_sign(int a, int j) {
    // VTK_HEXAHEDRON: (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1)
    return j == 0 ? (((a & 3) == 1 || (a & 3) == 2) ? 1 : -1)
                  : (j == 1 ? (((a & 3) >= 2) ? 1 : -1) : ((a >= 4) ? 1 : -1));
}

__host__ __device__ constexpr double hex_xi(int q, int j) { return ((q >> j) & 1) ? kGauss : -kGauss; }

// d N_a / d xi_j at Gauss point q
__host__ __device__ constexpr double hex_dN(int a, int q, int j) {
    return j == 0 ? 0.125 * hex_sign(a, 0) * (1.0 + hex_sign(a, 1) * hex_xi(q, 1)) *
                        (1.0 + hex_sign(a, 2) * hex_xi(q, 2))
           : j == 1 ? 0.125 * hex_sign(a, 1) * (1.0 + hex_sign(a, 0) * hex_xi(q, 0)) *
                          (1.0 + hex_sign(a, 2) * hex_xi(q, 2))
                    : 0.125 * hex_sign(a, 2) * (1.0 + hex_sign(a, 0) * hex_xi(q, 0)) *
                          (1.0 + hex_sign(a, 1) * hex_xi(q, 1));
}

// the same gradients as a table in constant memory, for a rolled loop over
// the Gauss points (all lanes read the same entry: a broadcast)
template <typename T>
struct HexDN {
    T v[8][7][3];  // [point][node 1..7][reference direction]
};
template <typename T>
__host__ __device__ constexpr HexDN<T> make_hex_dn() {
    HexDN<T> t{};
    for (int q = 0; q < 8; ++q)
        for (int a = 0; a < 7; ++a)
            for (int j = 0; j < 3; ++j) t.v[q][a][j] = (T)hex_dN(a + 1, q, j);
    return t;
}
static __constant__ HexDN<float> c_hex_dn_f = make_hex_dn<float>();
static __constant__ HexDN<double> c_hex_dn_d = make_hex_dn<double>();
template <typename T>
__device__ __forceinline__ T hex_dn(int q, int a, int j) {
    if constexpr (sizeof(T) == 4)
        return c_hex_dn_f.v[q][a][j];
    else
        return c_hex_dn_d.v[q][a][j];
}

// ---------------------------------------------------------------------------
// quadrature-point work, shared by P1 and Q1
// ---------------------------------------------------------------------------
// Per-lane partial sums of element scalars over a tile (s0: energy or vKv;
// s1: the energy's roundoff scale; ninv: quadrature points with J <= 0).
// FP64 calls add in double.  FP32 calls keep s0 as an unevaluated float pair
// hi + lo updated by Knuth's TwoSum, an error-free transformation, so the pair
// holds the lane's sum to about 2^-46 relative before it is widened to double
// once per tile; s1, a magnitude estimate, is a plain float sum.
// (hi, lo) += x by Knuth's TwoSum (FP32, error-free)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}
// warp total of (hi, lo) pairs, a fixed butterfly; every lane ends with it
__device__ __forceinline__ void ff_warp_total(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, oh);
        lo += ol;
    }
}

template <typename T>
struct ScalarAcc;
template <>
struct ScalarAcc<double> {
    double s0 = 0, s1 = 0;
    int ninv = 0;
    __device__ __forceinline__ void add0(double x) { s0 += x; }
    __device__ __forceinline__ void add1(double x) { s1 += x; }
    __device__ __forceinline__ double total0() const { return s0; }
    __device__ __forceinline__ double total1() const { return s1; }
};
template <>
struct ScalarAcc<float> {
    float hi = 0.f, lo = 0.f, s1 = 0.f;
    int ninv = 0;
    __device__ __forceinline__ void add0(float x) { ff_add(hi, lo, x); }
    __device__ __forceinline__ void add1(float x) { s1 += x; }
    __device__ __forceinline__ double total0() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ double total1() const { return (double)s1; }
};

template <int D, class V>
__device__ __forceinline__ void outer_sum(const V (*du)[D], const V (*g)[D], int n, V (&H)[D][D]) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            V s = du[0][i] * g[0][j];
            for (int a = 1; a < n; ++a) s = vfma(du[a][i], g[a][j], s);
            H[i][j] = s;
        }
}

// Given H (and dF), the gradients g of the NM1 non-reference nodes, w detJ
// and the moduli, accumulate contributions f[a] for those nodes (f[NM1] is the
// reference node for the block diagonal) and the scalar sums.  `valid` has a
// bit per lane-vector component that holds a real element.
// Per-element coefficients of the neural constitutive model (unscaled):
// the shifted network value, its roundoff scale, and NcmCoef's derivatives
template <int D, class V>
struct NcmElem {
    V C0, Cs;
    NcmCoef<D, V> d;
};

template <int OP, int D, int NM1, class V, bool NCM = false, bool LIN = false>
__device__ __forceinline__ void qp_work(const V (&H)[D][D], const V (&dF)[D][D], const V (&g)[NM1][D],
                                        V wdJ, V mu, V lam, int valid, V (&f)[NM1 + 1][6],
                                        ScalarAcc<typename VT<V>::S>& acc, bool scal, double (&gmu)[2],
                                        double (&glam)[2], int& inv, const NcmElem<D, V>* ncm = nullptr,
                                        typename VT<V>::S* ninv = nullptr, const typename VT<V>::S* lv = nullptr) {
    using S = typename VT<V>::S;
    constexpr int N = VT<V>::N;
    static_assert(!NCM || N == 1, "the neural constitutive model runs one element per lane");
    static_assert(!LIN || (N == 1 && OP == OP_HVP), "the stored linearisation serves the scalar HVP");
    if constexpr (LIN) {
        // dP = w mu dF + w (mu - lambda ln J) F^-T dF^T F^-T + w lambda tr(F^-1 dF) F^-T
        // from the stored F^-T and scaled moduli (zero for empty or inverted lanes)
        V FiT[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) FiT[i][j] = lv[i * D + j];
        const V wmu = lv[9], c1 = lv[10], wlam = lv[11];
        V trA = FiT[0][0] * dF[0][0];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (i + j > 0) trA = vfma(FiT[i][j], dF[i][j], trA);
        V M[D][D];  // dF^T F^-T
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                V t = dF[0][a] * FiT[0][j];
#pragma unroll
                for (int l = 1; l < D; ++l) t = vfma(dF[l][a], FiT[l][j], t);
                M[a][j] = t;
            }
        const V c2 = wlam * trA;
        V P[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                V B = FiT[i][0] * M[0][j];
#pragma unroll
                for (int a = 1; a < D; ++a) B = vfma(FiT[i][a], M[a][j], B);
                P[i][j] = vfma(c2, FiT[i][j], vfma(c1, B, wmu * dF[i][j]));
            }
        if (scal) {  // dP : dF
            V e = P[0][0] * dF[0][0];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j)
                    if (i + j > 0) e = vfma(P[i][j], dF[i][j], e);
            acc.add0(vsel(valid, e, S(0)));
        }
#pragma unroll
        for (int a = 0; a < NM1; ++a)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                V t = f[a][i];
#pragma unroll
                for (int j = 0; j < D; ++j) t = vfma(P[i][j], g[a][j], t);
                f[a][i] = t;
            }
        return;
    }
    Kin<D, V> k;
    kinematics<D, V>(H, k);
    if constexpr (OP == OP_NCM_INV) {
        static_assert(N == 1, "scalar lanes");
        if (valid & 1) {
            ninv[0] = vfma(splat<V>(S(2)), k.trH, k.HH);  // I1 - 3 = 2 tr H + H : H
            ninv[1] = k.Jm1;
        }
        return;
    }
    const int bad = valid & ~k.ok;
    if (bad) {
        inv |= bad;
        acc.ninv += __popc(bad);
    }
    const int good = valid & k.ok;
    wdJ = vsel(good, wdJ, S(0));  // inverted or empty halves contribute nothing
    if constexpr (OP == OP_LINEARIZE) {
        static_assert(N == 1, "scalar lanes");
        // every lane writes (16-byte stores): empty and inverted lanes get
        // zero moduli; 2D uses the first four of the nine F^-T slots
        S o[kLinVals];
#pragma unroll
        for (int q = 0; q < 9; ++q) o[q] = S(0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) o[i * D + j] = (i == j) ? k.G[i][j] + S(1) : k.G[i][j];
        o[9] = wdJ * mu;
        o[10] = wdJ * (mu - lam * k.lnJ);
        o[11] = wdJ * lam;
        if constexpr (sizeof(S) == 4) {
#pragma unroll
            for (int q = 0; q < kLinVals / 4; ++q)
                reinterpret_cast<float4*>(ninv)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < kLinVals / 2; ++q)
                reinterpret_cast<double2*>(ninv)[q] = make_double2(o[2 * q], o[2 * q + 1]);
        }
        return;
    }
    // the network's coefficients scaled by w det J (zero for bad lanes)
    NcmCoef<D, V> nc{};
    if constexpr (NCM) {
        nc.C2 = wdJ * ncm->d.C2;
        nc.C3 = wdJ * ncm->d.C3;
        nc.C11 = wdJ * ncm->d.C11;
        nc.C12 = wdJ * ncm->d.C12;
        nc.C22 = wdJ * ncm->d.C22;
    }
    if constexpr (OP == OP_ENERGY) {
        V psi, sc;
        density<D, V>(k, mu, lam, psi, sc);
        if constexpr (NCM) {
            psi = psi + ncm->C0;
            sc = sc + ncm->Cs;
        }
        // select, not multiply: a lane without an element (degenerate Q1
        // geometry) may carry a non-finite density
        const V a = vsel(good, wdJ * psi, S(0)), b = vsel(good, wdJ * sc, S(0));
#pragma unroll
        for (int c = 0; c < N; ++c) {
            acc.add0(vcomp(a, c));
            acc.add1(vcomp(b, c));
        }
    } else if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
        // P and dP are linear in (mu, lambda): w detJ folds into the moduli
        const V wmu = wdJ * mu, wlam = wdJ * lam;
        V P[D][D];
        if constexpr (OP == OP_RESIDUAL) {
            if constexpr (NCM)
                stress_ncm<D, V>(H, k, wmu, wlam, nc, P);
            else
                stress<D, V>(H, k, wmu, wlam, P);
        } else {
            if constexpr (NCM)
                tangent_ncm<D, V>(H, dF, k, wmu, wlam, nc, P);
            else
                tangent<D, V>(dF, k, wmu, wlam, P);
            if (scal) {  // w detJ dP : dF
                V e = P[0][0] * dF[0][0];
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j)
                        if (i + j > 0) e = vfma(P[i][j], dF[i][j], e);
                e = vsel(good, e, S(0));
#pragma unroll
                for (int c = 0; c < N; ++c) acc.add0(vcomp(e, c));
            }
        }
#pragma unroll
        for (int a = 0; a < NM1; ++a)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                V s = f[a][i];
#pragma unroll
                for (int j = 0; j < D; ++j) s = vfma(P[i][j], g[a][j], s);
                f[a][i] = s;
            }
    } else if constexpr (OP == OP_BLOCKDIAG) {
        // K_aa = wdJ [mu |g0|^2 I + (mu - lam lnJ + lam) gp gp^T], gp = F^-T g0
        const V c = wdJ * vfma(lam, splat<V>(S(1)) - k.lnJ, mu);
        const V m = wdJ * mu;
#pragma unroll
        for (int a = 0; a <= NM1; ++a) {
            V g0[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (a < NM1) {
                    g0[j] = g[a][j];
                } else {
                    V s = -g[0][j];
#pragma unroll
                    for (int b = 1; b < NM1; ++b) s = s - g[b][j];
                    g0[j] = s;
                }
            }
            V gp[D];
            V n2 = g0[0] * g0[0];
#pragma unroll
            for (int i = 1; i < D; ++i) n2 = vfma(g0[i], g0[i], n2);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                V s = g0[i];
#pragma unroll
                for (int j = 0; j < D; ++j) s = vfma(k.G[i][j], g0[j], s);
                gp[i] = s;
            }
            const V mn = m * n2;
            if constexpr (D == 3) {
                f[a][0] = f[a][0] + vfma(c * gp[0], gp[0], mn);
                f[a][1] = f[a][1] + vfma(c * gp[1], gp[1], mn);
                f[a][2] = f[a][2] + vfma(c * gp[2], gp[2], mn);
                f[a][3] = vfma(c * gp[0], gp[1], f[a][3]);
                f[a][4] = vfma(c * gp[0], gp[2], f[a][4]);
                f[a][5] = vfma(c * gp[1], gp[2], f[a][5]);
            } else {
                f[a][0] = f[a][0] + vfma(c * gp[0], gp[0], mn);
                f[a][1] = f[a][1] + vfma(c * gp[1], gp[1], mn);
                f[a][2] = vfma(c * gp[0], gp[1], f[a][2]);
            }
            if constexpr (NCM) block_ncm<D, V>(H, k, g0, gp, nc, f[a]);
        }
    } else if constexpr (OP == OP_PVJP) {
        // dP/dmu : grad a = (H - G) : grad a ; dP/dlam : grad a = lnJ (I + G) : grad a
        V sm = splat<V>(S(0)), sl = splat<V>(S(0));
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                sm = vfma(H[i][j] - k.G[i][j], dF[i][j], sm);
                sl = vfma(k.G[i][j], dF[i][j], sl);
                if (i == j) sl = sl + dF[i][j];
            }
        const V a = wdJ * sm, b = wdJ * k.lnJ * sl;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            gmu[c] += vget(a, c);
            glam[c] += vget(b, c);
        }
    }
}

template <int N, int ET, typename T>
struct Packer;
template <int ET, typename T>
struct Packer<1, ET, T> {
    __device__ __forceinline__ static T ed(const Half<ET, T>* hs, int j) { return hs[0].ed[j]; }
};
template <int ET, typename T>
struct Packer<2, ET, T> {
    __device__ __forceinline__ static F2 ed(const Half<ET, T>* hs, int j) {
        return mk2((float)hs[0].ed[j], (float)hs[1].ed[j]);
    }
};

// element of a round pair / single: gather, compute, return contributions
// Q1 Gauss point of the stored linearisation.  With J = dx/dxi, physical
// gradients J^-T dN/dxi and dF = dFr J^-1 (dFr = sum_a dv_a (x) dN_a/dxi),
// the nodal forces det J dP J^-T dN_a/dxi need
//   Q = det J dP J^-T = s1 dFr C + s2 A dFr^T A + s3 (A : dFr) A,
// A = F^-T J^-T, C = J^-1 J^-T, s1 = det J mu, s2 = det J (mu - lambda ln J),
// s3 = det J lambda (the tangent dP of the Neo-Hookean law, Sec. 2.1), and
// Q : dFr = det J dP : dF.
template <typename T>
__device__ __forceinline__ void hex_linearize_point(const T (&H)[3][3], const T (&Ji)[3][3], T detJ, T mu, T lam,
                                                    int valid, int& inv, ScalarAcc<T>& acc, T* dst) {
    Kin<3, T> k;
    kinematics<3, T>(H, k);
    const int bad = valid & ~k.ok;
    if (bad) {
        inv |= bad;
        acc.ninv += __popc(bad);
    }
    const bool good = (valid & k.ok) & 1;  // empty and inverted points store zeros
    T o[kHexLinVals];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T a = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) a = fma(k.G[i][l] + (i == l ? T(1) : T(0)), Ji[j][l], a);
            o[3 * i + j] = good ? a : T(0);
        }
    auto cij = [&](int i, int j) {
        T c = Ji[i][0] * Ji[j][0];
        c = fma(Ji[i][1], Ji[j][1], c);
        c = fma(Ji[i][2], Ji[j][2], c);
        return good ? c : T(0);
    };
    o[9] = cij(0, 0), o[10] = cij(1, 1), o[11] = cij(2, 2), o[12] = cij(0, 1), o[13] = cij(0, 2), o[14] = cij(1, 2);
    o[15] = good ? detJ * mu : T(0);
    o[16] = good ? detJ * (mu - lam * k.lnJ) : T(0);
    o[17] = good ? detJ * lam : T(0);
    o[18] = o[19] = T(0);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < kHexLinVals / 4; ++c)
            reinterpret_cast<float4*>(dst)[c * 32] = make_float4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < kHexLinVals / 2; ++c)
            reinterpret_cast<double2*>(dst)[c * 32] = make_double2(o[2 * c], o[2 * c + 1]);
    }
}

// src: the lane's first chunk of the point in the shared-memory stage
template <typename T>
__device__ __forceinline__ void hex_lin_point(const T (&dv)[7][3], const T (&gr)[7][3], const T* src, int valid,
                                              bool scal, ScalarAcc<T>& acc, T (&fr)[8][6]) {
    T w[kHexLinVals];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < kHexLinVals / 4; ++c) {
            const float4 t = reinterpret_cast<const float4*>(src)[c * 32];
            w[4 * c] = t.x, w[4 * c + 1] = t.y, w[4 * c + 2] = t.z, w[4 * c + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < kHexLinVals / 2; ++c) {
            const double2 t = reinterpret_cast<const double2*>(src)[c * 32];
            w[2 * c] = t.x, w[2 * c + 1] = t.y;
        }
    }
    T A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = w[3 * i + j];
    const T C[3][3] = {{w[9], w[12], w[13]}, {w[12], w[10], w[14]}, {w[13], w[14], w[11]}};
    const T s1 = w[15], s2 = w[16], s3 = w[17];
    T dFr[3][3];
    outer_sum<3, T>(dv, gr, 7, dFr);
    T t = A[0][0] * dFr[0][0];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (i + j > 0) t = fma(A[i][j], dFr[i][j], t);
    T X[3][3];  // dFr^T A
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T x = dFr[0][a] * A[0][j];
            x = fma(dFr[1][a], A[1][j], x);
            X[a][j] = fma(dFr[2][a], A[2][j], x);
        }
    const T s3t = s3 * t;
    T Q[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T m = dFr[i][0] * C[0][j];
            m = fma(dFr[i][1], C[1][j], m);
            m = fma(dFr[i][2], C[2][j], m);
            T b = A[i][0] * X[0][j];
            b = fma(A[i][1], X[1][j], b);
            b = fma(A[i][2], X[2][j], b);
            Q[i][j] = fma(s3t, A[i][j], fma(s2, b, s1 * m));
        }
    if (scal) {  // det J dP : dF
        T e = Q[0][0] * dFr[0][0];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (i + j > 0) e = fma(Q[i][j], dFr[i][j], e);
        acc.add0((valid & 1) ? e : T(0));
    }
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T f = fr[a][i];
#pragma unroll
            for (int j = 0; j < 3; ++j) f = fma(Q[i][j], gr[a][j], f);
            fr[a][i] = f;
        }
}

template <int ET, typename T, int OP, class V, bool NCM = false, bool LIN = false>
__device__ __forceinline__ void element_work(const Half<ET, T>* hs, int valid, const T* sU, const T* sV,
                                             const T* sX, V (&f)[ElemT<ET>::NEN][6], ScalarAcc<T>& acc,
                                             bool scal, double (&gmu)[2], double (&glam)[2], int& inv,
                                             const NcmElem<ElemT<ET>::D, V>* ncm = nullptr, T* ninv = nullptr,
                                             const T* lv = nullptr, T* lbuf = nullptr) {
    using E = ElemT<ET>;
    using S = typename VT<V>::S;
    constexpr int D = E::D, NEN = E::NEN, VW = E::VW, NM1 = NEN - 1, NG = E::NG;
    constexpr int N = VT<V>::N;
    using PK = Packer<N, ET, T>;
    constexpr bool kNeedV = (OP == OP_HVP || OP == OP_PVJP);
    V ue[NEN][D], ve[NEN][D];
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
        T t0[4], t1[4];
        if constexpr (LIN) {  // the stored linearisation replaces u
#pragma unroll
            for (int c = 0; c < D; ++c) ue[a][c] = splat<V>(S(0));
        } else {
            lds_vec<VW, T>(sU, hs[0].cn[a], t0);
            if constexpr (N == 2) lds_vec<VW, T>(sU, hs[N - 1].cn[a], t1);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (N == 2)
                    ue[a][c] = mk2(t0[c], t1[c]);
                else
                    ue[a][c] = (V)t0[c];
            }
        }
        if constexpr (kNeedV) {
            lds_vec<VW, T>(sV, hs[0].cn[a], t0);
            if constexpr (N == 2) lds_vec<VW, T>(sV, hs[N - 1].cn[a], t1);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (N == 2)
                    ve[a][c] = mk2(t0[c], t1[c]);
                else
                    ve[a][c] = (V)t0[c];
            }
        }
    }
    const V mu = PK::ed(hs, NG);
    const V lam = PK::ed(hs, NG + 1);
#pragma unroll
    for (int a = 0; a < NEN; ++a)
#pragma unroll
        for (int c = 0; c < 6; ++c) f[a][c] = splat<V>(S(0));

    if constexpr (ET != 2) {
        // P1: reference node = last; grad N_a (a < NEN-1) and w detJ from the record
        V g[NM1][D];
#pragma unroll
        for (int a = 0; a < NM1; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) g[a][c] = PK::ed(hs, a * D + c);
        const V wdJ = PK::ed(hs, NG - 1);
        V du[NM1][D], dv[NM1][D];
#pragma unroll
        for (int a = 0; a < NM1; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                du[a][c] = ue[a][c] - ue[NM1][c];
                if constexpr (kNeedV) dv[a][c] = ve[a][c] - ve[NM1][c];
            }
        V H[D][D], dF[D][D];
        outer_sum<D, V>(du, g, NM1, H);
        if constexpr (kNeedV) {
            outer_sum<D, V>(dv, g, NM1, dF);
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) dF[i][j] = splat<V>(S(0));
        }
        V fq[NM1 + 1][6];
#pragma unroll
        for (int a = 0; a <= NM1; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c) fq[a][c] = splat<V>(S(0));
        qp_work<OP, D, NM1, V, NCM, LIN>(H, dF, g, wdJ, mu, lam, valid, fq, acc, scal, gmu, glam, inv, ncm, ninv, lv);
        if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                V s = -fq[0][c];
                f[0][c] = fq[0][c];
#pragma unroll
                for (int a = 1; a < NM1; ++a) {
                    f[a][c] = fq[a][c];
                    s = s - fq[a][c];
                }
                f[NM1][c] = s;
            }
        } else if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
            for (int a = 0; a <= NM1; ++a)
#pragma unroll
                for (int c = 0; c < 6; ++c) f[a][c] = fq[a][c];
        }
    } else {
        static_assert(!NCM && OP != OP_NCM_INV, "the neural constitutive model covers P1 elements");
        static_assert(!(LIN || OP == OP_LINEARIZE) || N == 1, "the stored linearisation runs one element per lane");
        // Q1: reference node 0; J rebuilt at each Gauss point (or read with
        // the point's stored linearisation)
        constexpr int kChunk = 16 / (int)sizeof(T), kNch = hex_lin_chunks<T>();
        V dx[NM1][D], du[NM1][D], dv[NM1][D];
        if constexpr (LIN) {
#pragma unroll
            for (int a = 1; a < NEN; ++a)
#pragma unroll
                for (int c = 0; c < D; ++c) dv[a - 1][c] = ve[a][c] - ve[0][c];
        } else {
            T x0[4];
            lds_vec<VW, T>(sX, hs[0].cn[0], x0);
#pragma unroll
            for (int a = 1; a < NEN; ++a) {
                T t[4];
                lds_vec<VW, T>(sX, hs[0].cn[a], t);
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    dx[a - 1][c] = (V)(t[c] - x0[c]);
                    du[a - 1][c] = ue[a][c] - ue[0][c];
                    if constexpr (kNeedV) dv[a - 1][c] = ve[a][c] - ve[0][c];
                }
            }
        }
        V fr[NEN][6];  // nodes 1..7, then node 0 (block diagonal)
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c) fr[a][c] = splat<V>(S(0));
        // the stored linearisation: this lane's chunks of point q (global,
        // lane-major) into stage q % kSt of the warp's ring by cp.async, one
        // commit group per point (empty groups keep the count uniform)
        constexpr int kSt = hex_lin_stages((int)sizeof(T));
        const int lane_ = threadIdx.x & 31;
        auto lin_issue = [&](int q) {
            if (q < 8) {
                T* dst = lbuf + ((q % kSt) * kNch * 32 + lane_) * kChunk;
                const T* src = lv + q * kNch * 32 * kChunk;
#pragma unroll
                for (int c = 0; c < kNch; ++c) cp_async_cg16(dst + c * 32 * kChunk, src + c * 32 * kChunk);
            }
            cp_async_commit();
        };
        if constexpr (LIN) {
#pragma unroll
            for (int q = 0; q < kSt - 1; ++q) lin_issue(q);
        }
        // One Gauss point.  The full HVP runs the points in a rolled loop
        // with the reference gradients read from constant memory (smaller
        // code and fewer registers: measured 766 -> 680 us on hex128); the
        // other operators keep the unrolled loop with compile-time
        // gradients (measured faster for them)
        constexpr bool kRoll = OP == OP_HVP && !LIN;
        auto point = [&](const int q) {
            V gr[NM1][D];
#pragma unroll
            for (int a = 0; a < NM1; ++a)
#pragma unroll
                for (int j = 0; j < D; ++j) gr[a][j] = kRoll ? (V)hex_dn<T>(q, a, j) : (V)hex_dN(a + 1, q, j);
            if constexpr (LIN) {
                lin_issue(q + kSt - 1);
                cp_async_wait_group<kSt - 1>();  // point q has landed
                hex_lin_point<T>(dv, gr, lbuf + ((q % kSt) * kNch * 32 + lane_) * kChunk, valid, scal, acc, fr);
                return;
            }
            V Jm[D][D];
            outer_sum<D, V>(dx, gr, NM1, Jm);
            const V c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
            const V c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
            const V c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
            const V detJ = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
            const V rd = vrcp(detJ);
            V Ji[3][3];
            Ji[0][0] = c00 * rd;
            Ji[1][0] = c01 * rd;
            Ji[2][0] = c02 * rd;
            Ji[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) * rd;
            Ji[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) * rd;
            Ji[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) * rd;
            Ji[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) * rd;
            Ji[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) * rd;
            Ji[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) * rd;
            V g[NM1][D];
#pragma unroll
            for (int a = 0; a < NM1; ++a)
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    V s = Ji[0][i] * gr[a][0];
#pragma unroll
                    for (int j = 1; j < D; ++j) s = vfma(Ji[j][i], gr[a][j], s);
                    g[a][i] = s;
                }
            V H[D][D], dF[D][D];
            outer_sum<D, V>(du, g, NM1, H);
            if constexpr (OP == OP_LINEARIZE) {
                hex_linearize_point<T>(H, Ji, detJ, mu, lam, valid, inv, acc, ninv + q * kNch * 32 * kChunk);
                return;
            }
            if constexpr (kNeedV) {
                outer_sum<D, V>(dv, g, NM1, dF);
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) dF[i][j] = splat<V>(S(0));
            }
            qp_work<OP, D, NM1, V>(H, dF, g, detJ, mu, lam, valid, fr, acc, scal, gmu, glam, inv);
        };
        if constexpr (kRoll) {
#pragma unroll 1
            for (int q = 0; q < 8; ++q) point(q);
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) point(q);
        }
        if constexpr (OP == OP_RESIDUAL || OP == OP_HVP) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                V s = -fr[0][c];
                f[1][c] = fr[0][c];
#pragma unroll
                for (int a = 1; a < NM1; ++a) {
                    f[a + 1][c] = fr[a][c];
                    s = s - fr[a][c];
                }
                f[0][c] = s;
            }
        } else if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                f[0][c] = fr[NM1][c];
#pragma unroll
                for (int a = 0; a < NM1; ++a) f[a + 1][c] = fr[a][c];
            }
        }
    }
}

// block-diagonal entries (packed symmetric) -> full D x D with the Dirichlet identity
template <int D, typename T>
__device__ __forceinline__ int write_block(T* out, int64_t g, const T* s, uint8_t m) {
    T Dm[D][D];
    if constexpr (D == 3) {
        Dm[0][0] = s[0];
        Dm[1][1] = s[1];
        Dm[2][2] = s[2];
        Dm[0][1] = Dm[1][0] = s[3];
        Dm[0][2] = Dm[2][0] = s[4];
        Dm[1][2] = Dm[2][1] = s[5];
    } else {
        Dm[0][0] = s[0];
        Dm[1][1] = s[1];
        Dm[0][1] = Dm[1][0] = s[2];
    }
    int fl = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            T x = Dm[a][b];
            if (((m >> a) & 1) || ((m >> b) & 1)) x = (a == b) ? T(1) : T(0);
            if (!finite_(x)) fl |= 2;
            out[(g * D + a) * D + b] = x;
        }
    return fl;
}

template <int D, typename T>
__device__ __forceinline__ int write_vec(T* out, int64_t g, const T* s, uint8_t m, unsigned flags) {
    int fl = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        T x = s[c];
        if ((flags & 1u) && ((m >> c) & 1)) x = T(0);
        if (!finite_(x)) fl |= 2;
        out[g * D + c] = x;
    }
    return fl;
}

// Neumaier step: (s, c) += x
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// Fixed-order FP64 reduction of the tile partials tile_red[t][0..2] by one
// block of nthreads threads: strided per-thread Neumaier sums, a warp
// butterfly on (sum, compensation), then the warps in order.  `scratch` holds
// 4 doubles per warp.  Returns the totals in thread 0.
__device__ __forceinline__ void reduce_tiles(const double* tile_red, int n_tiles, int nthreads,
                                             double* scratch, double& S0, double& S1, double& N) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double sum0 = 0, c0 = 0, sum1 = 0, c1 = 0, cnt = 0;
    for (int t = tid; t < n_tiles; t += nthreads) {
        neumaier(sum0, c0, __ldcg(tile_red + (int64_t)t * 4 + 0));
        neumaier(sum1, c1, __ldcg(tile_red + (int64_t)t * 4 + 1));
        cnt += __ldcg(tile_red + (int64_t)t * 4 + 2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, sum0, o);
        const double oc = __shfl_xor_sync(0xffffffffu, c0, o);
        const double ps = __shfl_xor_sync(0xffffffffu, sum1, o);
        const double pc = __shfl_xor_sync(0xffffffffu, c1, o);
        const double on = __shfl_xor_sync(0xffffffffu, cnt, o);
        c0 += oc;
        neumaier(sum0, c0, os);
        c1 += pc;
        neumaier(sum1, c1, ps);
        cnt += on;
    }
    __syncthreads();
    if (lane == 0) {
        scratch[warp * 4 + 0] = sum0 + c0;
        scratch[warp * 4 + 1] = sum1 + c1;
        scratch[warp * 4 + 2] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        double a0 = 0, k0 = 0, a1 = 0, k1 = 0, n = 0;
        for (int w = 0; w < nthreads / 32; ++w) {
            neumaier(a0, k0, scratch[w * 4 + 0]);
            neumaier(a1, k1, scratch[w * 4 + 1]);
            n += scratch[w * 4 + 2];
        }
        S0 = a0 + k0;
        S1 = a1 + k1;
        N = n;
    }
}

// ---------------------------------------------------------------------------
// the tile kernel (persistent: CTA c runs tiles c, c + G, c + 2G, ...)
//
// Per tile: [nodes of this tile ready: fix-ups, zero accumulators] -> rounds
// (the records stream through the warp's ring, which runs ahead across tile
// boundaries; after its first round each thread issues cp.async gathers of
// the NEXT tile's nodal values into the other node buffer) -> combine and
// write -> bulk copy of the node ids / slots / masks of the tile after next.
// So a tile's node gathers overlap the previous tile's element work.
// ---------------------------------------------------------------------------
constexpr int kEmptyLane = 0xFFFF;  // local id of an empty lane (the planner's kNoNode)

// NCM: the neural constitutive model's terms from p.ncm_coef (P1 only).
// LIN: the HVP from the linearisation p.lin stored by OP_LINEARIZE at the
// same state (P1, Neo-Hookean; no u gather, no F, F^-1 or ln J)
template <int ET, typename T, int OP, bool NCM, bool LIN>
__device__ __forceinline__ void tile_body(const KParams& p) {
    using E = ElemT<ET>;
    constexpr int D = E::D, NEN = E::NEN, VW = E::VW;
    constexpr int NR = rounds_per_iter(ET, (int)sizeof(T), OP, LIN);
    constexpr bool kPacked =
        (FEM_PAIR_FP32 && ET != 2 && sizeof(T) == 4 && !NCM && !LIN && OP != OP_NCM_INV && OP != OP_LINEARIZE);
    static_assert(!LIN || (OP == OP_HVP && !NCM), "the stored linearisation serves the Neo-Hookean HVP");
    using V = typename std::conditional<kPacked, F2, T>::type;
    constexpr bool kNeedV = (OP == OP_HVP || OP == OP_PVJP);
    constexpr bool kNeedAcc = (OP == OP_RESIDUAL || OP == OP_HVP || OP == OP_BLOCKDIAG);
    extern __shared__ __align__(128) unsigned char smem[];

    const int G = gridDim.x, cta = blockIdx.x;
    const int n_my = (p.n_tiles > cta) ? (p.n_tiles - cta + G - 1) / G : 0;
    if (n_my == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SmemLayout L = smem_layout(ET, (int)sizeof(T), OP, p.max_nlp, p.rec_bytes, LIN);
    const int AW = L.aw;
    T* sAcc = reinterpret_cast<T*>(smem + L.off_acc);
    double* sRed = reinterpret_cast<double*>(smem + L.off_red);
    int* sFlag = reinterpret_cast<int*>(smem + L.off_red + kWarps * 4 * 8);
    int4* tab = reinterpret_cast<int4*>(smem + L.off_tab);  // (node begin, padded count, round begin, rounds)
    uint8_t* ring = smem + L.off_ring + warp * kStages * L.stage_bytes;
    uint64_t* rbar = reinterpret_cast<uint64_t*>(smem + L.off_bar) + warp * kStages;
    auto buf = [&](int b) { return smem + (b ? L.off_buf1 : L.off_buf0); };

    const T* gu = static_cast<const T*>(p.u);
    const T* gv = static_cast<const T*>(p.v);
    const T* gx = static_cast<const T*>(p.X);
    const T mu0 = (T)p.mu0, lam0 = (T)p.lam0;
    // the HVP's fused vKv only when the caller asked for it
    const bool want_scalar = (OP == OP_ENERGY) || (OP == OP_HVP && (p.out_scalar != nullptr || p.vkv_tiles));
    int flags_local = 0;

    // 0. tile table and barriers
    for (int i = tid; i < n_my; i += kThreads) {
        const int t = cta + i * G;
        const int64_t n0 = p.tile_node_ptr[t], n1 = p.tile_node_ptr[t + 1];
        const int r0 = p.tile_round_ptr[t], r1 = p.tile_round_ptr[t + 1];
        tab[i] = make_int4((int)n0, (int)(n1 - n0), r0, r1 - r0);
    }
    if (tid == 0) {
        for (int k = 0; k < kWarps * kStages; ++k)
            mbar_init(reinterpret_cast<uint64_t*>(smem + L.off_bar) + k, 1);
        *sFlag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // Node metadata (global id, partial slot, Dirichlet bits) of the current
    // and the next tile, in registers: node j = tid + kThreads k for k < kMeta
    // (nodes of larger tiles beyond that are read from global memory where
    // used).  The next tile's metadata is loaded a tile ahead of its use.
    constexpr int kMeta = (ET == 2) ? 1 : 4;
    struct Meta {
        int g[kMeta], s[kMeta];
        uint32_t m;
    };
    auto load_meta = [&](int i, Meta& M) {
        const int4 tb = tab[i];
        M.m = 0u;
#pragma unroll
        for (int k = 0; k < kMeta; ++k) {
            const int j = tid + kThreads * k;
            M.g[k] = -1;
            M.s[k] = -1;
            if (j < tb.y) {
                M.g[k] = __ldg(p.node_gid + tb.x + j);
                M.s[k] = __ldg(p.node_slot + tb.x + j);
                M.m |= (uint32_t)__ldg(p.node_mask_local + tb.x + j) << (8 * k);
            }
        }
    };
    // gather tile i's nodal values into buffer i & 1 (all threads, cp.async)
    auto gather = [&](int i, const Meta& M) {
        const int4 tb = tab[i];
        unsigned char* B = buf(i & 1);
        T* bu = reinterpret_cast<T*>(B + L.off_u);
        T* bv = reinterpret_cast<T*>(B + L.off_v);
        T* bx = reinterpret_cast<T*>(B + L.off_x);
        auto one = [&](int j, int64_t g) {
            if (g < 0) return;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (!LIN) cp_async<sizeof(T)>(bu + j * VW + c, gu + g * D + c);
                if constexpr (kNeedV) cp_async<sizeof(T)>(bv + j * VW + c, gv + g * D + c);
                if constexpr (ET == 2 && !LIN) cp_async<sizeof(T)>(bx + j * VW + c, gx + g * D + c);
            }
        };
#pragma unroll
        for (int k = 0; k < kMeta; ++k)
            if (tid + kThreads * k < tb.y) one(tid + kThreads * k, M.g[k]);
        for (int j = tid + kThreads * kMeta; j < tb.y; j += kThreads) one(j, __ldg(p.node_gid + tb.x + j));
        cp_async_commit();
    };

    // ring producer (lane 0 of each warp): the warp's iterations of its
    // tiles, in order, kStages ahead of the consumer
    auto my_range = [&](int i, int& r0, int& n) {
        const int4 tb = tab[i];
        const int R = tb.w;
        r0 = tb.z + warp * (R / kWarps) + min(warp, R % kWarps);
        n = R / kWarps + (warp < R % kWarps ? 1 : 0);
    };
    int pi = 0, pit = 0, p_r0 = 0, p_n = 0, p_slot = 0, issued = 0;
    my_range(0, p_r0, p_n);
    auto issue_next = [&]() {
        while (pit * NR >= p_n) {  // next tile with rounds for this warp
            if (++pi >= n_my) return;
            pit = 0;
            my_range(pi, p_r0, p_n);
        }
        const int nrec = min(NR, p_n - pit * NR);
        const int64_t r0 = p_r0 + pit * NR;
        if constexpr (LIN && ET != 2)  // the rounds' records, then their stored linearisation
            bulk_load2_hint(ring + p_slot * L.stage_bytes, p.rec + r0 * p.rec_bytes, (uint32_t)(nrec * p.rec_bytes),
                            ring + p_slot * L.stage_bytes + NR * p.rec_bytes,
                            static_cast<const unsigned char*>(p.lin) + r0 * 32 * kLinVals * (int64_t)sizeof(T),
                            (uint32_t)(nrec * 32 * kLinVals * (int)sizeof(T)), &rbar[p_slot], l2_evict_first());
        else
            bulk_load(ring + p_slot * L.stage_bytes, p.rec + r0 * p.rec_bytes, (uint32_t)(nrec * p.rec_bytes),
                      &rbar[p_slot]);

        p_slot = (p_slot + 1 == kStages) ? 0 : p_slot + 1;
        ++pit;
        ++issued;
    };

    // 1. start: metadata of the first two tiles, the ring, tile 0's gathers.
    // Under a programmatic dependent launch the CTAs start while the previous
    // kernel drains: up to here only mesh data (plan, metadata) is read, and
    // nothing an earlier kernel writes is touched before the wait.
    Meta cur, nxt;
    load_meta(0, cur);
    if (n_my > 1) load_meta(1, nxt);
    grid_dependency_wait();
    if (p.skip != nullptr && *p.skip != 0) return;  // uniform: set by an earlier kernel
    if (lane == 0)
        for (int k = 0; k < kStages; ++k) issue_next();
    gather(0, cur);

    int consumed = 0, c_slot = 0;
    uint32_t c_phase = 0;
    bool timed_out = false;
    int inv = 0;
    for (int i = 0; i < n_my; ++i) {
        const int t = cta + i * G;
        unsigned char* B = buf(i & 1);
        T* sU = reinterpret_cast<T*>(B + L.off_u);
        T* sV = reinterpret_cast<T*>(B + L.off_v);
        T* sX = reinterpret_cast<T*>(B + L.off_x);
        const int nlp = tab[i].y;
        const int64_t nbase = tab[i].x;

        cp_async_wait_all();
        __syncthreads();
        // 2. fix-ups of the gathered values; zero the accumulators
        auto fixup = [&](int j, int g, uint32_t m) {
            if (g < 0) return;
            bool fin = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (!LIN) fin = fin && finite_(sU[j * VW + c]);
                if constexpr (kNeedV) {
                    if (OP == OP_HVP && (p.flags & 2u) && ((m >> c) & 1)) sV[j * VW + c] = T(0);
                    fin = fin && finite_(sV[j * VW + c]);
                }
            }
            if (!fin) flags_local |= 2;
        };
#pragma unroll
        for (int k = 0; k < kMeta; ++k)
            if (tid + kThreads * k < nlp) fixup(tid + kThreads * k, cur.g[k], (cur.m >> (8 * k)) & 0xffu);
        for (int j = tid + kThreads * kMeta; j < nlp; j += kThreads)
            fixup(j, __ldg(p.node_gid + nbase + j), __ldg(p.node_mask_local + nbase + j));
        if constexpr (kNeedAcc) {
            int4* z = reinterpret_cast<int4*>(sAcc);
            const int nz = align16(kWarps * nlp * AW * (int)sizeof(T)) / 16;
            for (int j = tid; j < nz; j += kThreads) z[j] = make_int4(0, 0, 0, 0);
        }
        __syncthreads();

        // 3. rounds
        int my_r0, my_n;
        my_range(i, my_r0, my_n);
        const int n_it = (my_n + NR - 1) / NR;
        T* myAcc = sAcc + (int64_t)warp * nlp * AW;
        ScalarAcc<T> acc;
        bool gathered = (i + 1 >= n_my);
        for (int it = 0; it < n_it && !timed_out; ++it) {
            const int s = c_slot;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&rbar[s], c_phase))) {  // warp-uniform
                timed_out = true;
                break;
            }
            ++consumed;
            if (++c_slot == kStages) {
                c_slot = 0;
                c_phase ^= 1u;
            }
            const int k0 = it * NR;
            const uint8_t* st = ring + s * L.stage_bytes;
            Half<ET, T> hs[NR];
            int valid = 0;
#pragma unroll
            for (int h = 0; h < NR; ++h) {
                const bool ok = read_half<ET, T>(st + h * p.rec_bytes, lane, k0 + h < my_n, p, mu0, lam0, hs[h]);
                valid |= ok ? (1 << h) : 0;
            }
            // the stored linearisation of this lane's elements, read before the
            // stage is refilled (16-byte lane-major chunks: conflict-free)
            T linv[LIN && ET != 2 ? NR : 1][kLinVals];
            if constexpr (LIN && ET != 2) {
#pragma unroll
                for (int h = 0; h < NR; ++h) {
                    const bool here = k0 + h < my_n;
                    const unsigned char* src = st + NR * p.rec_bytes + (size_t)(h * 32 + lane) * kLinVals * sizeof(T);
                    if constexpr (sizeof(T) == 4) {
#pragma unroll
                        for (int q = 0; q < kLinVals / 4; ++q) {
                            const float4 w = here ? reinterpret_cast<const float4*>(src)[q] : make_float4(0, 0, 0, 0);
                            linv[h][4 * q] = w.x, linv[h][4 * q + 1] = w.y;
                            linv[h][4 * q + 2] = w.z, linv[h][4 * q + 3] = w.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < kLinVals / 2; ++q) {
                            const double2 w = here ? reinterpret_cast<const double2*>(src)[q] : make_double2(0, 0);
                            linv[h][2 * q] = w.x, linv[h][2 * q + 1] = w.y;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_next();
            }
            if (!gathered) {  // the next tile's nodes, spread over all threads
                gather(i + 1, nxt);
                gathered = true;
            }
            // element contributions: f[h] for round k0 + h (scalar), or both
            // rounds packed in f[0] (FP32x2 pairs)
            constexpr int NF = kPacked ? 1 : NR;
            V f[NF][NEN][6] = {};
            auto fc = [&](int h, int a, int c) -> T {
                if constexpr (kPacked)
                    return vcomp(f[0][a][c], h);
                else
                    return (T)f[h][a][c];
            };
            auto scatter = [&](int h) {
#pragma unroll
                for (int a = 0; a < NEN; ++a) {
                    const int n = hs[h].cn[a];
                    if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
                        for (int c = 0; c < (D == 3 ? 6 : 3); ++c) myAcc[n * AW + c] += fc(h, a, c);
                    } else {
                        T cur[4];
                        lds_vec<VW, T>(myAcc, n, cur);
#pragma unroll
                        for (int c = 0; c < D; ++c) cur[c] += fc(h, a, c);
                        // a fresh value in the padding lane keeps the store one
                        // 16-byte access: storing back the loaded padding lets
                        // the compiler narrow it to 8 + 4 bytes, and a 4-byte
                        // store at a 16-byte stride hits a bank 4 times
                        if constexpr (VW > D) cur[VW - 1] = T(0);
                        sts_vec<VW, T>(myAcc, n, cur);
                    }
                }
            };
            double gmu[NR][2] = {}, glam[NR][2] = {};
            if constexpr (kPacked) {
                if (valid) element_work<ET, T, OP, V>(hs, valid, sU, sV, sX, f[0], acc, want_scalar, gmu[0], glam[0], inv);
            } else {
                // warp-uniform: the round is present; lanes without an element
                // compute on zero geometry and skip the scatter
#pragma unroll
                for (int h = 0; h < NR; ++h)
                    if (k0 + h < my_n) {
                        // this lane's element in record order (round * 32 + lane)
                        const int64_t rec = (int64_t)(my_r0 + k0 + h) * 32 + lane;
                        NcmElem<D, V> ne{};
                        if constexpr (NCM) {
                            T c[8];
                            const T* src = static_cast<const T*>(p.ncm_coef) + rec * 8;
                            if constexpr (sizeof(T) == 4) {
                                const float4 c0 = __ldg(reinterpret_cast<const float4*>(src));
                                const float4 c1 = __ldg(reinterpret_cast<const float4*>(src) + 1);
                                c[0] = c0.x, c[1] = c0.y, c[2] = c0.z, c[3] = c0.w;
                                c[4] = c1.x, c[5] = c1.y, c[6] = c1.z, c[7] = c1.w;
                            } else {
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const double2 cj = __ldg(reinterpret_cast<const double2*>(src) + j);
                                    c[2 * j] = cj.x, c[2 * j + 1] = cj.y;
                                }
                            }
                            ne.C0 = c[0], ne.Cs = c[1];
                            ne.d.C2 = c[2], ne.d.C3 = c[3], ne.d.C11 = c[4], ne.d.C12 = c[5], ne.d.C22 = c[6];
                        }
                        T* ninv = nullptr;
                        if constexpr (OP == OP_NCM_INV) ninv = static_cast<T*>(p.ncm_inv) + rec * 2;
                        // Q1: the lane's first 16-byte chunk of the round (lane-major)
                        const int64_t hex_lin = ((int64_t)(my_r0 + k0 + h) * 8 * hex_lin_chunks<T>() * 32 + lane) *
                                                (16 / (int64_t)sizeof(T));
                        if constexpr (OP == OP_LINEARIZE)
                            ninv = static_cast<T*>(p.lin) + (ET == 2 ? hex_lin : rec * kLinVals);
                        const T* lv = nullptr;
                        if constexpr (LIN) lv = ET == 2 ? static_cast<const T*>(p.lin) + hex_lin : linv[h];
                        T* lbuf = reinterpret_cast<T*>(smem + L.off_lin) +
                                  (size_t)warp * hex_lin_stages((int)sizeof(T)) * 32 * kHexLinVals;
                        element_work<ET, T, OP, V, NCM, LIN>(&hs[h], (valid >> h) & 1, sU, sV, sX,
                                                             f[NF == 1 ? 0 : h], acc, want_scalar, gmu[h], glam[h],
                                                             inv, &ne, ninv, lv, lbuf);
                    }
            }
            if constexpr (OP == OP_PVJP) {
#pragma unroll
                for (int h = 0; h < NR; ++h)
                    if (valid & (1 << h)) {
                        const int e = p.round_elem[(int64_t)(my_r0 + k0 + h) * 32 + lane];
                        const double gm = kPacked ? gmu[0][h] : gmu[h][0];
                        const double gl = kPacked ? glam[0][h] : glam[h][0];
                        if (p.out_mu) p.out_mu[e] = gm;
                        if (p.out_lam) p.out_lam[e] = gl;
                    }
            }
            if constexpr (kNeedAcc) {
#pragma unroll
                for (int h = 0; h < NR; ++h) {
                    if (h > 0) __syncwarp();  // round k0+h-1 lands first: rounds may share nodes
                    if (valid & (1 << h)) scatter(h);
                }
            }
            __syncwarp();
        }
        if (!gathered && !timed_out) gather(i + 1, nxt);  // a warp without rounds in this tile

        // 4. scalar partial of this tile (fixed order).  The HVP's vKv: one
        // sum, kept in FP32 pairs through the warps for FP32 calls (FP64
        // instructions issue at a small fraction of the FP32 rate here)
        if (OP == OP_HVP && want_scalar) {
            if constexpr (sizeof(T) == 4) {
                float hi = acc.hi, lo = acc.lo;
                ff_warp_total(hi, lo);
                if (lane == 0) {
                    reinterpret_cast<float*>(sRed)[warp * 2 + 0] = hi;
                    reinterpret_cast<float*>(sRed)[warp * 2 + 1] = lo;
                }
            } else {
                double s0 = acc.total0();
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                if (lane == 0) sRed[warp * 4] = s0;
            }
        }
        if (OP == OP_ENERGY && want_scalar) {
            double s0 = acc.total0(), s1 = acc.total1(), s2 = (double)acc.ninv;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            if (lane == 0) {
                sRed[warp * 4 + 0] = s0;
                sRed[warp * 4 + 1] = s1;
                sRed[warp * 4 + 2] = s2;
            }
        }
        __syncthreads();
        if constexpr (OP == OP_HVP) {
            if (tid == 0 && want_scalar) {
                if constexpr (sizeof(T) == 4) {
                    float hi = 0.f, lo = 0.f;
                    for (int w = 0; w < kWarps; ++w) {
                        ff_add(hi, lo, reinterpret_cast<const float*>(sRed)[w * 2 + 0]);
                        lo += reinterpret_cast<const float*>(sRed)[w * 2 + 1];
                    }
                    reinterpret_cast<float*>(p.tile_red + (int64_t)t * 4)[0] = hi;
                    reinterpret_cast<float*>(p.tile_red + (int64_t)t * 4)[1] = lo;
                } else {
                    double a0 = 0;
                    for (int w = 0; w < kWarps; ++w) a0 += sRed[w * 4];
                    p.tile_red[(int64_t)t * 4] = a0;
                }
            }
        }
        if constexpr (OP == OP_ENERGY) {
            if (tid == 0) {
                double a0 = 0, a1 = 0, a2 = 0;
                for (int w = 0; w < kWarps; ++w) {
                    a0 += sRed[w * 4 + 0];
                    a1 += sRed[w * 4 + 1];
                    a2 += sRed[w * 4 + 2];
                }
                p.tile_red[(int64_t)t * 4 + 0] = a0;
                p.tile_red[(int64_t)t * 4 + 1] = a1;
                p.tile_red[(int64_t)t * 4 + 2] = a2;
            }
        }

        // 5. combine the warp copies; write private nodes and shared partials
        if constexpr (kNeedAcc) {
            T* part = static_cast<T*>(p.partial);
            T* out = static_cast<T*>(p.out);
            auto combine = [&](int j, int g, int slot, uint32_t msk) {
                if (g < 0) return;
                T sum[6] = {0, 0, 0, 0, 0, 0};
                if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
                    for (int w = 0; w < kWarps; ++w)
                        for (int c = 0; c < AW; ++c) sum[c] += sAcc[((int64_t)w * nlp + j) * AW + c];
                } else {
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) {
                        T tv[4];
                        lds_vec<VW, T>(sAcc + (int64_t)w * nlp * VW, j, tv);
#pragma unroll
                        for (int c = 0; c < VW; ++c) sum[c] += tv[c];
                    }
                }
                if (slot < 0) {
                    if constexpr (OP == OP_BLOCKDIAG)
                        flags_local |= write_block<D, T>(out, g, sum, (uint8_t)msk);
                    else
                        flags_local |= write_vec<D, T>(out, g, sum, (uint8_t)msk, p.flags);
                } else if constexpr (OP == OP_BLOCKDIAG) {
                    for (int c = 0; c < AW; ++c) part[(int64_t)slot * AW + c] = sum[c];
                } else {
                    sts_vec<VW, T>(part, slot, sum);  // one node vector per slot
                }
            };
#pragma unroll
            for (int k = 0; k < kMeta; ++k)
                if (tid + kThreads * k < nlp)
                    combine(tid + kThreads * k, cur.g[k], cur.s[k], (cur.m >> (8 * k)) & 0xffu);
            for (int j = tid + kThreads * kMeta; j < nlp; j += kThreads)
                combine(j, __ldg(p.node_gid + nbase + j), __ldg(p.node_slot + nbase + j),
                        __ldg(p.node_mask_local + nbase + j));
        }
        __syncthreads();
        // 6. the next tile's metadata becomes current; load tile i + 2's
        cur = nxt;
        if (i + 2 < n_my) load_meta(i + 2, nxt);
    }
    if (timed_out) flags_local |= 4;
    // drain the copies still in flight before the CTA may exit
    if (lane == 0)
        for (int j = consumed; j < issued; ++j)
            mbar_wait_bounded(&rbar[j % kStages], (uint32_t)((j / kStages) & 1));
    cp_async_wait_all();
    if (inv) flags_local |= 1;
    {
        const int wf = __reduce_or_sync(0xffffffffu, flags_local);
        if (lane == 0 && wf) atomicOr(sFlag, wf);
    }

    // 7. the HVP's vKv: the last CTA adds the tile partials in tile order
    // (FP32 pairs for FP32 calls, doubles for FP64 calls)
    if (OP == OP_HVP && p.out_scalar != nullptr) {
        __shared__ int s_last_h;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_last_h = (atomicAdd(p.tile_counter, 1u) == (unsigned)G - 1u);
        }
        __syncthreads();
        if (s_last_h) {
            __threadfence();
            if constexpr (sizeof(T) == 4) {
                float hi = 0.f, lo = 0.f;
                for (int t = tid; t < p.n_tiles; t += kThreads) {
                    const float2 x = __ldcg(reinterpret_cast<const float2*>(p.tile_red + (int64_t)t * 4));
                    ff_add(hi, lo, x.x);
                    lo += x.y;
                }
                ff_warp_total(hi, lo);
                if (lane == 0) {
                    reinterpret_cast<float*>(sRed)[warp * 2 + 0] = hi;
                    reinterpret_cast<float*>(sRed)[warp * 2 + 1] = lo;
                }
                __syncthreads();
                if (tid == 0) {
                    float h = 0.f, l = 0.f;
                    for (int w = 0; w < kWarps; ++w) {
                        ff_add(h, l, reinterpret_cast<const float*>(sRed)[w * 2 + 0]);
                        l += reinterpret_cast<const float*>(sRed)[w * 2 + 1];
                    }
                    p.out_scalar[0] = (double)h + (double)l;
                    *p.tile_counter = 0u;
                }
            } else {
                double a = 0.0;
                for (int t = tid; t < p.n_tiles; t += kThreads) a += __ldcg(p.tile_red + (int64_t)t * 4);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) sRed[warp * 4] = a;
                __syncthreads();
                if (tid == 0) {
                    double h = 0.0;
                    for (int w = 0; w < kWarps; ++w) h += sRed[w * 4];
                    p.out_scalar[0] = h;
                    *p.tile_counter = 0u;
                }
            }
        }
    }
    // 7. energy: the last CTA reduces the tile partials in tile order
    if constexpr (OP == OP_ENERGY) {
        __shared__ int s_last;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_last = (atomicAdd(p.tile_counter, 1u) == (unsigned)G - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double S0 = 0, S1 = 0, N = 0;
            reduce_tiles(p.tile_red, p.n_tiles, kThreads, sRed, S0, S1, N);
            if (tid == 0) {
                p.out_scalar[0] = N > 0 ? __longlong_as_double(0x7ff0000000000000ll) : S0;
                p.out_scalar[1] = S1;
                p.out_scalar[2] = N;
                p.out_scalar[3] = 0.0;
                *p.tile_counter = 0u;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && *sFlag) atomicOr(p.status, *sFlag);
}

template <int ET, typename T, int OP, bool NCM = false, bool LIN = false>
__global__ void __launch_bounds__(kThreads) tile_kernel(const KParams p) {
    tile_body<ET, T, OP, NCM, LIN>(p);
}

// the FP32 HVP from a stored linearisation: two rounds per iteration within
// the registers of four CTAs per SM (one round: within those of five)
template <int ET>
__global__ void __launch_bounds__(kThreads, FEM_DUAL_LIN ? 4 : 5) tile_kernel_lin(const KParams p) {
    tile_body<ET, float, OP_HVP, false, true>(p);
}

// FP32 Q1 operators with a register budget of FEM_HEX_MINB CTAs per SM
#ifndef FEM_HEX_MINB
#define FEM_HEX_MINB 2
#endif
template <int OP, bool LIN = false>
__global__ void __launch_bounds__(kThreads, FEM_HEX_MINB) tile_kernel_hex(const KParams p) {
    tile_body<2, float, OP, false, LIN>(p);
}

// ---------------------------------------------------------------------------
// finalize: each shared node's partial slots summed in slot order, and nodes
// of no element
// ---------------------------------------------------------------------------
template <int D, typename T, int OP>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const KParams p) {
    constexpr int VW = D == 2 ? 2 : 4;
    constexpr int AW = (OP == OP_BLOCKDIAG) ? (D == 2 ? 4 : 6) : VW;
    const int total = p.n_shared + p.n_orphans;
    const int j0 = blockIdx.x * kFinThreads + threadIdx.x;
    // the shared-node records are mesh data: the first one is loaded while
    // the tile kernel drains
    int4 inf = make_int4(0, 0, 0, 0);
    if (j0 < p.n_shared) inf = __ldg(p.shared_info + j0);
    grid_dependency_wait();  // the tile kernel's writes are visible past this point
    if (p.skip != nullptr && *p.skip != 0) return;
    const T* part = static_cast<const T*>(p.partial);
    T* out = static_cast<T*>(p.out);
    int fl = 0;
    for (int j = j0; j < total; j += gridDim.x * kFinThreads) {
        if (j < p.n_shared) {
            if (j != j0) inf = __ldg(p.shared_info + j);
            const int s0 = inf.x, s1 = inf.y, g = inf.z;
            const uint8_t m = (uint8_t)inf.w;
            T sum[6] = {0, 0, 0, 0, 0, 0};
            // slots in batches of kFinBatch: the loads of a batch are issued
            // together, then added in slot order
            constexpr int kFinBatch = 4;
            for (int q0 = s0; q0 < s1; q0 += kFinBatch) {
                T t[kFinBatch][AW > 4 ? AW : 4];
#pragma unroll
                for (int b = 0; b < kFinBatch; ++b) {
                    if (q0 + b >= s1) break;
                    if constexpr (OP == OP_BLOCKDIAG) {
#pragma unroll
                        for (int c = 0; c < AW; ++c) t[b][c] = part[(int64_t)(q0 + b) * AW + c];
                    } else {
                        lds_vec<VW, T>(part, q0 + b, t[b]);
                    }
                }
#pragma unroll
                for (int b = 0; b < kFinBatch; ++b) {
                    if (q0 + b >= s1) break;
#pragma unroll
                    for (int c = 0; c < AW; ++c) sum[c] += t[b][c];
                }
            }
            if constexpr (OP == OP_BLOCKDIAG)
                fl |= write_block<D, T>(out, g, sum, m);
            else
                fl |= write_vec<D, T>(out, g, sum, m, p.flags);
        } else {
            const int g = p.orphans[j - p.n_shared];
            const T zero[6] = {0, 0, 0, 0, 0, 0};
            if constexpr (OP == OP_BLOCKDIAG)
                write_block<D, T>(out, g, zero, (uint8_t)0x7);
            else
                write_vec<D, T>(out, g, zero, 0, 0u);
        }
    }
    if (fl) atomicOr(p.status, fl);
}

}  // namespace fem
