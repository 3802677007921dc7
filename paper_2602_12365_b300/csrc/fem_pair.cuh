// Pair kernels: the FP32 residual and HVP of P1 elements (Algorithm 1:
// gather, field gradient, Neo-Hookean stress or tangent action, scatter)
// with every lane computing TWO elements at once, one from each of two rounds,
// in the two halves of the paired FP32 instructions of sm_100+ (fma.rn.f32x2:
// one issue slot for two FMAs).  The tet residual and HVP are bound by
// instruction issue, not by HBM (at the HBM floor an SM can issue about 330
// warp instructions per round of 32 elements, the one-element kernel needs
// about 500), and the element arithmetic is ~60 % of their instructions: two
// elements per instruction remove most of it.
//
// Work decomposition as the tile kernel (fem_kernels.cuh): one CTA per tile,
// kWarps warps, per-warp accumulator copies, node buffers double-buffered
// and gathered a tile ahead, shared nodes through partial slots and the
// finalize kernel, every sum in a fixed order (bitwise reproducible).  What
// differs:
//   records  a PAIR record holds two rounds of a warp's range (A = rounds
//            r0 + 2k, B = r0 + 2k + 1; an odd range ends with an empty B):
//            per lane one 16-byte chunk of node ids (A's then B's), then the
//            geometry as (A, B) pairs in 16-byte chunks (grad N and w det J:
//            pair j of a lane at chunk j / 2), then (mu_A, mu_B, lam_A,
//            lam_B) when the moduli vary per element.  A 16-byte load gives
//            two ready pairs, so the paired arithmetic needs no packing.
//   empty    lanes without an element name a dummy node (index max_nlp, zero
//            in both node buffers) and carry zero geometry, so they compute
//            zero contributions with no branch; the dummy accumulator entry
//            is never read back.
//   math     one straight-line block per pair: no data-dependent branch (the
//            branch-free FP32 logarithm of fem_vec.cuh).
// The scatter adds A's contributions (low halves) for all lanes, then B's
// (high halves): the lanes of one round share no node, and the warp
// synchronises between the two rounds.
//
// Four kernels share the body: the residual and the HVP at (u, v); the
// linearisation pass (OP_LINEARIZE, at u, written as (A, B) pairs in
// pair-record order, lane-major 16-byte chunks); and the HVP from that
// stored linearisation (LIN), which is the PCG's operator.  The stored form
// holds, per element, b_a = F^-T grad N_a for the vertices but the last, the
// scaled metric w mu grad N_a . grad N_b, w (mu - lambda ln J) and w lambda.
// With dF = sum_b dv_b (x) grad N_b (dv_b = v_b - v_last) the tangent of
// the Neo-Hookean stress applied to grad N_a then reads
//   w dP grad N_a = sum_b (w mu grad N_a . grad N_b) dv_b
//                 + w (mu - lambda ln J) sum_b (b_a . dv_b) b_b
//                 + w lambda (sum_b b_b . dv_b) b_a,
// so the LIN HVP needs neither u, F, F^-1 and ln J nor the record's
// geometry: its ring stage carries the record's node ids and the lin block
// only.  The HVPs can leave per-tile FP32-pair partials of v^T K v
// (vkv_tiles) for the PCG's fused dot product.
#pragma once
#include "fem_kernels.cuh"

namespace fem {

// pairs of a tile of R rounds: warp w runs the pair_rounds(R, w) consecutive
// rounds after those of the warps before it (the tile kernel's split) as
// pair_count(R, w) pairs, starting at pair pair_first(R, w) of the tile
__host__ __device__ inline int pair_rounds(int R, int w) { return R / kWarps + (w < R % kWarps ? 1 : 0); }
__host__ __device__ inline int pair_count(int R, int w) { return (pair_rounds(R, w) + 1) / 2; }
__host__ __device__ inline int pair_first(int R, int w) {
    int f = 0;
    for (int v = 0; v < w; ++v) f += pair_count(R, v);
    return f;
}

template <int ET>
struct PairT;
template <>
struct PairT<0> {  // P1 triangle, plane strain: grad N_0, grad N_1, w det J
    static constexpr int D = 2, NEN = 3, NG = 5, NCH = 3;
};
template <>
struct PairT<1> {  // P1 tetrahedron: grad N_0..grad N_2, w det J
    static constexpr int D = 3, NEN = 4, NG = 10, NCH = 5;
};

// bytes of one pair record: ids, geometry pairs, optional moduli
__host__ __device__ constexpr int pair_rec_bytes(int et, bool mat) {
    return 32 * 16 * (1 + (et == 0 ? 3 : 5) + (mat ? 1 : 0));
}

// lin block of one pair record, in 16-byte chunks of two (A, B) pairs per
// lane: b_a (D (NEN - 1) values), the metric's upper triangle, the two
// scaled moduli and one zero -- tet 9 + 6 + 2 + 1 = 18 values, 9 chunks;
// triangle 4 + 3 + 2 + 1 = 10 values, 5 chunks
__host__ __device__ constexpr int pair_lin_chunks(int et) { return et == 0 ? 5 : 9; }
__host__ __device__ constexpr int pair_lin_bytes(int et) { return 32 * 16 * pair_lin_chunks(et); }

// bytes of the pair record a kernel copies: the ids and the geometry, plus
// the moduli chunk when they vary per element; the HVP from the stored
// linearisation copies the ids chunk only (the lin block carries the rest)
__host__ __device__ constexpr int pair_copy_bytes(int et, bool mat, bool lin) {
    return lin ? 32 * 16 : pair_rec_bytes(et, mat);
}

struct PairLayout {
    int off_u, off_v, buf_bytes, off_buf0, off_buf1, off_acc, acc_stride, off_red, off_tab, off_tabp, off_ring,
        stage_bytes, off_bar, total;
};

// node buffers hold max_nlp + 1 entries (the last is the dummy node); u
// unless LIN, v for the HVPs, accumulators unless OP_LINEARIZE
__host__ __device__ inline PairLayout pair_layout(int et, int op, bool lin, int max_nlp, int copy_bytes) {
    const int vw = et == 0 ? 2 : 4;
    const int nodes = max_nlp + 1;
    const int vec = align16(nodes * vw * 4);
    const bool has_u = !lin, has_v = op == OP_HVP, has_acc = op != OP_LINEARIZE;
    PairLayout L;
    L.off_u = 0;
    L.off_v = has_u ? vec : 0;
    L.buf_bytes = (has_u ? vec : 0) + (has_v ? vec : 0);
    L.off_buf0 = 0;
    L.off_buf1 = L.buf_bytes;
    int o = 2 * L.buf_bytes;
    // per-warp accumulator copies at a 16-byte stride (acc_stride floats),
    // so that every copy starts on a 16-byte boundary for vector stores
    L.off_acc = o;
    L.acc_stride = has_acc ? vec / 4 : 0;
    o += kWarps * L.acc_stride * 4;
    L.off_red = o;  // the CTA's status flags, then the warps' v^T K v pairs
    o = align16(o + 16 + kWarps * 8);
    L.off_tab = o;
    o = align16(o + kMaxTilesPerCta * 16);
    L.off_tabp = o;
    o = align16(o + kMaxTilesPerCta * 4);
    L.stage_bytes = copy_bytes + (lin ? pair_lin_bytes(et) : 0);
    L.off_ring = o = align16(o);
    o += kWarps * L.stage_bytes;
    L.off_bar = o = align16(o);
    o += kWarps * 8;
    L.total = align16(o);
    return L;
}

// pair j of a lane from its geometry chunks
__device__ __forceinline__ F2 pair_of(const float4 (&gc)[5], int j) {
    const float4 c = gc[j >> 1];
    return (j & 1) ? mk2(c.z, c.w) : mk2(c.x, c.y);
}

template <int ET, int OP, bool LIN>
__device__ __forceinline__ void pair_body(const KParams& p) {
    using PT = PairT<ET>;
    constexpr int D = PT::D, NEN = PT::NEN, NM1 = NEN - 1, NG = PT::NG, NCH = PT::NCH;
    constexpr int VW = D == 2 ? 2 : 4;
    constexpr bool kLinz = OP == OP_LINEARIZE;     // writes the linearisation
    constexpr bool kHvp = OP == OP_HVP;
    constexpr bool kNeedU = !LIN, kNeedV = kHvp, kAcc = !kLinz;
    constexpr int NLC = pair_lin_chunks(ET), kLinBytes = pair_lin_bytes(ET);
    constexpr int NMET = NM1 * (NM1 + 1) / 2;  // the metric's upper triangle
    static_assert(D * NM1 + NMET + 3 == 4 * NLC / 2, "the lin block: b_a, metric, two moduli, one zero");
    static_assert(OP == OP_RESIDUAL || OP == OP_HVP || OP == OP_LINEARIZE, "pair kernels: residual, HVP, linearise");
    static_assert(!LIN || kHvp, "the stored linearisation serves the HVP");
    extern __shared__ __align__(128) unsigned char smem[];

    const int G = gridDim.x, cta = blockIdx.x;
    const int n_my = (p.n_tiles > cta) ? (p.n_tiles - cta + G - 1) / G : 0;
    if (n_my == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int copy_bytes = pair_copy_bytes(ET, p.has_mat != 0, LIN);
    const PairLayout L = pair_layout(ET, OP, LIN, p.max_nlp, copy_bytes);
    const int nodes = p.max_nlp + 1;
    float* sAcc = reinterpret_cast<float*>(smem + L.off_acc);
    int* sFlag = reinterpret_cast<int*>(smem + L.off_red);
    float* sRed = reinterpret_cast<float*>(smem + L.off_red + 16);  // per warp (hi, lo) of v^T K v
    int4* tab = reinterpret_cast<int4*>(smem + L.off_tab);  // (node begin, padded count, round begin, rounds)
    int* tabp = reinterpret_cast<int*>(smem + L.off_tabp);  // first pair record of the tile
    uint8_t* ring = smem + L.off_ring + warp * L.stage_bytes;
    uint64_t* rbar = reinterpret_cast<uint64_t*>(smem + L.off_bar) + warp;
    auto bufU = [&](int b) { return reinterpret_cast<float*>(smem + (b ? L.off_buf1 : L.off_buf0) + L.off_u); };
    auto bufV = [&](int b) { return reinterpret_cast<float*>(smem + (b ? L.off_buf1 : L.off_buf0) + L.off_v); };
    const float* gu = static_cast<const float*>(p.u);
    const float* gv = static_cast<const float*>(p.v);
    const float mu0 = (float)p.mu0, lam0 = (float)p.lam0;
    const bool want_vkv = kHvp && p.vkv_tiles != 0;
    int flags_local = 0;

    // 0. tile table, barriers, the dummy node (zero in both buffers)
    for (int i = tid; i < n_my; i += kThreads) {
        const int t = cta + i * G;
        const int64_t n0 = p.tile_node_ptr[t], n1 = p.tile_node_ptr[t + 1];
        const int r0 = p.tile_round_ptr[t], r1 = p.tile_round_ptr[t + 1];
        tab[i] = make_int4((int)n0, (int)(n1 - n0), r0, r1 - r0);
        tabp[i] = p.tile_pair_ptr[t];
    }
    if (tid == 0) {
        for (int k = 0; k < kWarps; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem + L.off_bar) + k, 1);
        *sFlag = 0;
        fence_mbar_init();
    }
    if (tid < 2 * VW) {
        const int b = tid / VW, c = tid % VW;
        if constexpr (kNeedU) bufU(b)[(nodes - 1) * VW + c] = 0.f;
        if constexpr (kNeedV) bufV(b)[(nodes - 1) * VW + c] = 0.f;
    }
    __syncthreads();

    // node metadata (global id, partial slot, Dirichlet bits) of the current
    // and the next tile in registers, a tile ahead of its use
    constexpr int kMeta = 4;
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
                if constexpr (kAcc) {
                    M.s[k] = __ldg(p.node_slot + tb.x + j);
                    M.m |= (uint32_t)__ldg(p.node_mask_local + tb.x + j) << (8 * k);
                }
            }
        }
    };
    // gather tile i's nodal values into buffer i & 1 (all threads, cp.async)
    auto gather = [&](int i, const Meta& M) {
        const int4 tb = tab[i];
        float* bu = bufU(i & 1);
        float* bv = bufV(i & 1);
        // the HVP's input mask is applied here: a masked component is stored
        // as zero instead of copied (so nothing rewrites the buffer later)
        const bool mask_in = kNeedV && (p.flags & 2u);
        auto one = [&](int j, int64_t g, uint32_t m) {
            if (g < 0) return;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (kNeedU) cp_async<4>(bu + j * VW + c, gu + g * D + c);
                if constexpr (kNeedV) {
                    if (mask_in && ((m >> c) & 1))
                        bv[j * VW + c] = 0.f;
                    else
                        cp_async<4>(bv + j * VW + c, gv + g * D + c);
                }
            }
        };
#pragma unroll
        for (int k = 0; k < kMeta; ++k)
            if (tid + kThreads * k < tb.y) one(tid + kThreads * k, M.g[k], (M.m >> (8 * k)) & 0xffu);
        for (int j = tid + kThreads * kMeta; j < tb.y; j += kThreads)
            one(j, __ldg(p.node_gid + tb.x + j), kNeedV ? __ldg(p.node_mask_local + tb.x + j) : 0u);
        cp_async_commit();
    };
    // this warp's pair records of tile i
    auto my_pairs = [&](int i, int& p0, int& np) {
        const int R = tab[i].w;
        p0 = tabp[i] + pair_first(R, warp);
        np = pair_count(R, warp);
    };
    // ring producer (lane 0): a cursor over the warp's pair records across
    // its tiles gives the next record index (-1 past the last); one record
    // (and, for LIN, its lin block) per copy, one stage per warp
    struct Cursor {
        int i, it, p0, np;
    };
    auto next_rec = [&](Cursor& q) -> int64_t {
        while (q.it >= q.np) {
            if (++q.i >= n_my) return -1;
            q.it = 0;
            my_pairs(q.i, q.p0, q.np);
        }
        return (int64_t)(q.p0 + q.it++);
    };
    Cursor cc{0, 0, 0, 0};
    my_pairs(0, cc.p0, cc.np);
    int issued = 0;
    const unsigned char* glin = static_cast<const unsigned char*>(p.lin);
    auto issue_next = [&]() {
        const int64_t r = next_rec(cc);
        if (r < 0) return;
        if constexpr (LIN)  // the record's ids chunk, then its lin block; read once: evict first
            bulk_load2_hint(ring, p.prec + r * p.prec_bytes, (uint32_t)copy_bytes, ring + copy_bytes,
                            glin + r * kLinBytes, (uint32_t)kLinBytes, rbar, l2_evict_first());
        else
            bulk_load(ring, p.prec + r * p.prec_bytes, (uint32_t)copy_bytes, rbar);
        ++issued;
    };

    // 1. start (up to the wait, only mesh data is read: programmatic
    // dependent launch)
    Meta cur, nxt;
    load_meta(0, cur);
    if (n_my > 1) load_meta(1, nxt);
    grid_dependency_wait();
    if (p.skip != nullptr && *p.skip != 0) return;
    if (lane == 0) issue_next();
    gather(0, cur);

    int consumed = 0;
    bool timed_out = false;
    int inv = 0;
    for (int i = 0; i < n_my; ++i) {
        const int t = cta + i * G;
        float* sU = bufU(i & 1);
        float* sV = bufV(i & 1);
        const int nlp = tab[i].y;
        const int64_t nbase = tab[i].x;
        // this tile's nodes have landed, and every warp is done with the
        // previous tile's accumulator copies (combined before this barrier)
        cp_async_wait_all();
        __syncthreads();
        // 2. the finite-input check (reads only) and each warp's own
        // accumulator copy zeroed: no further barrier before the rounds
        auto fixup = [&](int j, int g) {
            if (g < 0) return;
            bool fin = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (kNeedU) fin = fin && finite_(sU[j * VW + c]);
                if constexpr (kNeedV) fin = fin && finite_(sV[j * VW + c]);
            }
            if (!fin) flags_local |= 2;
        };
#pragma unroll
        for (int k = 0; k < kMeta; ++k)
            if (tid + kThreads * k < nlp) fixup(tid + kThreads * k, cur.g[k]);
        for (int j = tid + kThreads * kMeta; j < nlp; j += kThreads) fixup(j, __ldg(p.node_gid + nbase + j));
        if constexpr (kAcc) {
            float* myz = sAcc + (size_t)warp * L.acc_stride;
            float4* z = reinterpret_cast<float4*>(myz);
            const int nz = (nlp * VW + 3) / 4;
            for (int j = lane; j < nz; j += 32) z[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();

        // 3. pairs of rounds
        int p0, np;
        my_pairs(i, p0, np);
        float* myAcc = sAcc + (size_t)warp * L.acc_stride;
        bool gathered = (i + 1 >= n_my);
        float vk_hi = 0.f, vk_lo = 0.f;  // this lane's v^T K v over the tile (TwoSum pair)
        for (int k = 0; k < np && !timed_out; ++k) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(rbar, (uint32_t)(consumed & 1)))) {
                timed_out = true;  // warp-uniform
                break;
            }
            ++consumed;
            const uint8_t* st = ring;
            const uint4 cw = reinterpret_cast<const uint4*>(st)[lane];
            float4 gc[5];
#pragma unroll
            for (int c = 0; c < 5; ++c)
                gc[c] = (!LIN && c < NCH) ? reinterpret_cast<const float4*>(st + 512 * (1 + c))[lane]
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 mc = make_float4(mu0, mu0, lam0, lam0);
            if (!LIN && p.has_mat) mc = reinterpret_cast<const float4*>(st + 512 * (1 + NCH))[lane];
            float4 lc[LIN ? NLC : 1];
            if constexpr (LIN) {
#pragma unroll
                for (int c = 0; c < NLC; ++c) lc[c] = reinterpret_cast<const float4*>(st + copy_bytes + 512 * c)[lane];
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
            int ia[NEN], ib[NEN];
            if constexpr (NEN == 4) {
                ia[0] = cw.x & 0xffff, ia[1] = cw.x >> 16, ia[2] = cw.y & 0xffff, ia[3] = cw.y >> 16;
                ib[0] = cw.z & 0xffff, ib[1] = cw.z >> 16, ib[2] = cw.w & 0xffff, ib[3] = cw.w >> 16;
            } else {
                ia[0] = cw.x & 0xffff, ia[1] = cw.x >> 16, ia[2] = cw.y & 0xffff;
                ib[0] = cw.z & 0xffff, ib[1] = cw.z >> 16, ib[2] = cw.w & 0xffff;
            }
            // gather and differences against the reference (last) node: the
            // scalar differences land in the two halves of the pairs
            auto diffs = [&](const float* buf, F2 (&dd)[NM1][D]) {
                float ta[NEN][4], tb[NEN][4];
#pragma unroll
                for (int a = 0; a < NEN; ++a) {
                    lds_vec<VW, float>(buf, ia[a], ta[a]);
                    lds_vec<VW, float>(buf, ib[a], tb[a]);
                }
#pragma unroll
                for (int a = 0; a < NM1; ++a)
#pragma unroll
                    for (int c = 0; c < D; ++c) dd[a][c] = mk2(ta[a][c] - ta[NM1][c], tb[a][c] - tb[NM1][c]);
            };
            F2 g[NM1][D];  // grad N_a (zero for LIN, which reads no geometry)
#pragma unroll
            for (int a = 0; a < NM1; ++a)
#pragma unroll
                for (int c = 0; c < D; ++c) g[a][c] = pair_of(gc, a * D + c);
            F2 P[D][D];
            F2 dF[D][D];
            F2 dv[NM1][D];
            F2 f[NEN][D];  // forces on the vertices but the last (the last: minus their sum)
            if constexpr (kNeedV) diffs(sV, dv);
            if constexpr (kNeedV && !LIN) outer_sum<D, F2>(dv, g, NM1, dF);
            if constexpr (LIN) {
                // the forces from the stored b_a, metric and scaled moduli
                // (all zero for empty or inverted elements)
                auto lp = [&](int j) {
                    const float4 c = lc[j >> 1];
                    return (j & 1) ? mk2(c.z, c.w) : mk2(c.x, c.y);
                };
                F2 b[NM1][D];
#pragma unroll
                for (int a = 0; a < NM1; ++a)
#pragma unroll
                    for (int c = 0; c < D; ++c) b[a][c] = lp(a * D + c);
                F2 met[NM1][NM1];  // w mu grad N_a . grad N_b: diagonal, then (0,1), (0,2), (1,2)
                {
                    int q = D * NM1;
#pragma unroll
                    for (int a = 0; a < NM1; ++a) met[a][a] = lp(q++);
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int c = a + 1; c < NM1; ++c) met[a][c] = met[c][a] = lp(q++);
                }
                const F2 c1 = lp(D * NM1 + NMET), wlam = lp(D * NM1 + NMET + 1);
                F2 m[NM1][NM1];  // b_a . dv_c
#pragma unroll
                for (int a = 0; a < NM1; ++a)
#pragma unroll
                    for (int c = 0; c < NM1; ++c) {
                        F2 t2 = b[a][0] * dv[c][0];
#pragma unroll
                        for (int k = 1; k < D; ++k) t2 = vfma(b[a][k], dv[c][k], t2);
                        m[a][c] = t2;
                    }
                F2 tr = m[0][0];
#pragma unroll
                for (int a = 1; a < NM1; ++a) tr = tr + m[a][a];
                const F2 sl = wlam * tr;
#pragma unroll
                for (int a = 0; a < NM1; ++a) {
                    F2 n[NM1];
#pragma unroll
                    for (int c = 0; c < NM1; ++c) n[c] = c1 * m[a][c];
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        F2 t2 = sl * b[a][k];
#pragma unroll
                        for (int c = 0; c < NM1; ++c) t2 = vfma(met[a][c], dv[c][k], vfma(n[c], b[c][k], t2));
                        f[a][k] = t2;
                    }
                }
                if (want_vkv) {  // v^T K v of both halves: sum_a dv_a . f_a (the forces sum to zero)
                    F2 e = dv[0][0] * f[0][0];
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int k = 0; k < D; ++k)
                            if (a + k > 0) e = vfma(dv[a][k], f[a][k], e);
                    ff_add(vk_hi, vk_lo, e.v.x);
                    ff_add(vk_hi, vk_lo, e.v.y);
                }
            } else {
                F2 du[NM1][D];
                diffs(sU, du);
                F2 wdJ = pair_of(gc, NG - 1);
                F2 H[D][D];
                outer_sum<D, F2>(du, g, NM1, H);
                Kin<D, F2> kin;
                kinematics<D, F2, true>(H, kin);
                const int bad = 3 & ~kin.ok;  // empty halves have H = 0, J = 1
                inv |= bad;
                wdJ = vsel(kin.ok, wdJ, 0.f);  // inverted halves contribute nothing
                const F2 mu = mk2(mc.x, mc.y), lam = mk2(mc.z, mc.w);
                const F2 wmu = wdJ * mu, wlam = wdJ * lam;
                if constexpr (kLinz) {
                    // b_a = F^-T grad N_a, the metric w mu grad N_a . grad N_b,
                    // w (mu - lambda ln J), w lambda and a zero, as the pair's
                    // lin block (lane-major chunks); inverted halves store zeros
                    F2 o[2 * NLC];
                    int q = 0;
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            // row c of F^-T = I + G, applied to grad N_a
                            F2 t2 = g[a][c];
#pragma unroll
                            for (int k = 0; k < D; ++k) t2 = vfma(kin.G[c][k], g[a][k], t2);
                            o[q++] = vsel(kin.ok, t2, 0.f);
                        }
                    auto dot_g = [&](int a, int c) {
                        F2 t2 = g[a][0] * g[c][0];
#pragma unroll
                        for (int k = 1; k < D; ++k) t2 = vfma(g[a][k], g[c][k], t2);
                        return wmu * t2;
                    };
#pragma unroll
                    for (int a = 0; a < NM1; ++a) o[q++] = dot_g(a, a);
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int c = a + 1; c < NM1; ++c) o[q++] = dot_g(a, c);
                    o[q++] = wdJ * (mu - lam * kin.lnJ);
                    o[q++] = wlam;
                    o[q++] = mk2(0.f, 0.f);
                    float4* dst = reinterpret_cast<float4*>(static_cast<unsigned char*>(p.lin) +
                                                            (int64_t)(p0 + k) * kLinBytes) + lane;
#pragma unroll
                    for (int c = 0; c < NLC; ++c)
                        dst[32 * c] = make_float4(o[2 * c].v.x, o[2 * c].v.y, o[2 * c + 1].v.x, o[2 * c + 1].v.y);
                } else if constexpr (kHvp) {
                    tangent<D, F2>(dF, kin, wmu, wlam, P);
                } else {
                    stress<D, F2>(H, kin, wmu, wlam, P);
                }
            }
            if constexpr (kAcc) {
                if constexpr (!LIN) {
                    if constexpr (kHvp) {
                        if (want_vkv) {  // w dP : dF of both halves
                            F2 e = P[0][0] * dF[0][0];
#pragma unroll
                            for (int i2 = 0; i2 < D; ++i2)
#pragma unroll
                                for (int j = 0; j < D; ++j)
                                    if (i2 + j > 0) e = vfma(P[i2][j], dF[i2][j], e);
                            ff_add(vk_hi, vk_lo, e.v.x);
                            ff_add(vk_hi, vk_lo, e.v.y);
                        }
                    }
#pragma unroll
                    for (int a = 0; a < NM1; ++a)
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            F2 s2 = P[c][0] * g[a][0];
#pragma unroll
                            for (int j = 1; j < D; ++j) s2 = vfma(P[c][j], g[a][j], s2);
                            f[a][c] = s2;
                        }
                }
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    F2 s2 = -f[0][c];
#pragma unroll
                    for (int a = 1; a < NM1; ++a) s2 = s2 - f[a][c];
                    f[NM1][c] = s2;
                }
                // scatter round A (low halves), then round B (high halves).  The
                // lanes of one round hit distinct nodes of the warp's own copy, so
                // the adds of a node come in round order (fixed, reproducible)
                auto scatter = [&](const int (&id)[NEN], int h) {
#pragma unroll
                    for (int a = 0; a < NEN; ++a) {
                        float cur4[4];
                        lds_vec<VW, float>(myAcc, id[a], cur4);
#pragma unroll
                        for (int c = 0; c < D; ++c) cur4[c] += vcomp(f[a][c], h);
                        // a fresh padding value keeps the store one 16-byte access
                        if constexpr (VW > D) cur4[VW - 1] = 0.f;
                        sts_vec<VW, float>(myAcc, id[a], cur4);
                    }
                };
                scatter(ia, 0);
                __syncwarp();
                scatter(ib, 1);
                __syncwarp();
            }  // kAcc
        }
        if (!gathered && !timed_out) gather(i + 1, nxt);  // a warp without pairs in this tile

        // 4. the tile's v^T K v partial: warps in order, FP32 pairs
        if (want_vkv) {
            ff_warp_total(vk_hi, vk_lo);
            if (lane == 0) {
                sRed[warp * 2 + 0] = vk_hi;
                sRed[warp * 2 + 1] = vk_lo;
            }
        }
        __syncthreads();
        if (want_vkv && tid == 0) {
            float hi = 0.f, lo = 0.f;
            for (int w = 0; w < kWarps; ++w) {
                ff_add(hi, lo, sRed[w * 2 + 0]);
                lo += sRed[w * 2 + 1];
            }
            reinterpret_cast<float*>(p.tile_red + (int64_t)t * 4)[0] = hi;
            reinterpret_cast<float*>(p.tile_red + (int64_t)t * 4)[1] = lo;
        }

        // 5. combine the warp copies in warp order; private nodes to the
        // output, shared nodes to their partial slot
        if constexpr (kAcc) {
            float* part = static_cast<float*>(p.partial);
            float* out = static_cast<float*>(p.out);
            auto combine = [&](int j, int g, int slot, uint32_t msk) {
                if (g < 0) return;
                float sum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    float tv[4];
                    lds_vec<VW, float>(sAcc + (size_t)w * L.acc_stride, j, tv);
#pragma unroll
                    for (int c = 0; c < VW; ++c) sum[c] += tv[c];
                }
                if (slot < 0)
                    flags_local |= write_vec<D, float>(out, g, sum, (uint8_t)msk, p.flags);
                else
                    sts_vec<VW, float>(part, slot, sum);
            };
#pragma unroll
            for (int k = 0; k < kMeta; ++k)
                if (tid + kThreads * k < nlp) combine(tid + kThreads * k, cur.g[k], cur.s[k], (cur.m >> (8 * k)) & 0xffu);
            for (int j = tid + kThreads * kMeta; j < nlp; j += kThreads)
                combine(j, __ldg(p.node_gid + nbase + j), __ldg(p.node_slot + nbase + j),
                        __ldg(p.node_mask_local + nbase + j));
        }
        // (the next tile's first barrier also orders these reads of the
        // copies before their zeroing)
        cur = nxt;
        if (i + 2 < n_my) load_meta(i + 2, nxt);
    }
    if (timed_out) flags_local |= 4;
    // drain the copy still in flight before the CTA may exit
    if (lane == 0)
        for (int j = consumed; j < issued; ++j) mbar_wait_bounded(rbar, (uint32_t)(j & 1));
    cp_async_wait_all();
    if (inv) flags_local |= 1;
    {
        const int wf = __reduce_or_sync(0xffffffffu, flags_local);
        if (lane == 0 && wf) atomicOr(sFlag, wf);
    }
    __syncthreads();
    if (tid == 0 && *sFlag) atomicOr(p.status, *sFlag);
}

// four CTAs of kThreads per SM: at most 128 registers per thread
template <int ET, int OP, bool LIN = false>
__global__ void __launch_bounds__(kThreads, 4) pair_kernel(const KParams p) {
    pair_body<ET, OP, LIN>(p);
}

}  // namespace fem
