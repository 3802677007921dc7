// Host-side two-level partition (see fem_plan.h).  Pure C++, no CUDA, so the
// colouring can be built and checked on a machine without a GPU.
#include "fem_plan.h"

#include <algorithm>
#include <cstring>
#include <numeric>

namespace fem {

namespace {

using u128 = unsigned __int128;

struct Centroids {
    int dim;
    std::vector<double> c;  // [n_el*dim]
    double at(int64_t e, int k) const { return c[(size_t)e * dim + k]; }
};

// Recursive coordinate bisection: split [lo, hi) of idx at a position that
// keeps every leaf at most T elements, along the axis of largest centroid
// extent; ties broken by element id so the split is unique.
void rcb(const Centroids& C, std::vector<int32_t>& idx, int64_t lo, int64_t hi, int T,
         std::vector<int64_t>& leaves) {
    int64_t n = hi - lo;
    int64_t k = (n + T - 1) / T;
    if (k <= 1) {
        leaves.push_back(hi);
        return;
    }
    int64_t kl = k / 2;
    int64_t nl = n * kl / k;
    int axis = 0;
    double best = -1.0;
    for (int a = 0; a < C.dim; ++a) {
        double mn = 1e300, mx = -1e300;
        for (int64_t i = lo; i < hi; ++i) {
            double v = C.at(idx[i], a);
            mn = std::min(mn, v);
            mx = std::max(mx, v);
        }
        if (mx - mn > best) {
            best = mx - mn;
            axis = a;
        }
    }
    auto cmp = [&](int32_t a, int32_t b) {
        double va = C.at(a, axis), vb = C.at(b, axis);
        return va < vb || (va == vb && a < b);
    };
    std::nth_element(idx.begin() + lo, idx.begin() + lo + nl, idx.begin() + hi, cmp);
    rcb(C, idx, lo, lo + nl, T, leaves);
    rcb(C, idx, lo + nl, hi, T, leaves);
}

inline int lowest_zero(u128 m) {
    uint64_t lo = (uint64_t)m, hi = (uint64_t)(m >> 64);
    if (~lo) return __builtin_ctzll(~lo);
    if (~hi) return 64 + __builtin_ctzll(~hi);
    return 128;
}

// First-fit colouring with capacity kRound of the tile's elements, visited in
// `order`.  local[e*n_en + a] are tile-local node ids.  Returns the number of
// rounds (or kMaxRounds + 1 on overflow); round_of[i] is the round of element
// position i.
int colour_tile(const std::vector<int>& order, const std::vector<int>& local, int n_en,
                int n_local, std::vector<int>& round_of) {
    std::vector<u128> used(n_local, 0);
    u128 full = 0;
    int count[kMaxRounds] = {0};
    int n_rounds = 0;
    round_of.assign(order.size(), -1);
    for (int pos : order) {
        u128 m = full;
        for (int a = 0; a < n_en; ++a) m |= used[local[pos * n_en + a]];
        int r = lowest_zero(m);
        if (r >= kMaxRounds) return kMaxRounds + 1;
        round_of[pos] = r;
        u128 bit = (u128)1 << r;
        for (int a = 0; a < n_en; ++a) used[local[pos * n_en + a]] |= bit;
        if (++count[r] == kRound) full |= bit;
        n_rounds = std::max(n_rounds, r + 1);
    }
    return n_rounds;
}

}  // namespace

std::string build_plan(const MeshInput& in, Plan& P) {
    const int d = in.dim, ne = in.n_en;
    const int64_t NN = in.n_nodes, NE = in.n_el;
    P = Plan();
    P.dim = d;
    P.n_en = ne;
    P.n_en_pad = ne <= 4 ? 4 : 8;
    P.elem_type = in.elem_type;
    P.n_nodes = NN;
    P.n_el = NE;
    int T = in.tile_elems > 0 ? in.tile_elems : (in.elem_type == 2 ? 512 : 1024);
    P.tile_elems = T;
    if (NE <= 0 || NN <= 0) return "empty mesh";
    if (NE > INT32_MAX || NN > INT32_MAX) return "mesh too large for int32 ids";
    for (int64_t k = 0; k < NE * ne; ++k)
        if (in.conn[k] < 0 || in.conn[k] >= NN) return "connectivity references a node out of range";

    // centroids
    Centroids C{d, std::vector<double>((size_t)NE * d, 0.0)};
    for (int64_t e = 0; e < NE; ++e)
        for (int a = 0; a < ne; ++a)
            for (int k = 0; k < d; ++k)
                C.c[(size_t)e * d + k] += in.X[(size_t)in.conn[e * ne + a] * d + k] / ne;

    std::vector<int32_t> idx(NE);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<int64_t> leaves;
    rcb(C, idx, 0, NE, T, leaves);
    const int nt = (int)leaves.size();

    std::vector<int32_t> loc(NN, -1);
    std::vector<int32_t> tiles_of_node(NN, 0);
    P.tile_round_ptr.assign(1, 0);
    P.tile_node_ptr.assign(1, 0);

    int64_t start = 0;
    std::vector<int> local, order, order2, round_of, round_of2, valence;
    std::vector<int32_t> gids;
    for (int t = 0; t < nt; ++t) {
        int64_t end = leaves[t];
        int E = (int)(end - start);
        // local node numbering: ascending global id
        gids.clear();
        for (int64_t i = start; i < end; ++i)
            for (int a = 0; a < ne; ++a) gids.push_back(in.conn[(int64_t)idx[i] * ne + a]);
        std::sort(gids.begin(), gids.end());
        gids.erase(std::unique(gids.begin(), gids.end()), gids.end());
        int nl = (int)gids.size();
        if (nl > 65535) return "tile has more than 65535 nodes";
        for (int j = 0; j < nl; ++j) {
            loc[gids[j]] = j;
            tiles_of_node[gids[j]]++;
        }
        local.assign((size_t)E * ne, 0);
        valence.assign(nl, 0);
        for (int i = 0; i < E; ++i)
            for (int a = 0; a < ne; ++a) {
                int l = loc[in.conn[(int64_t)idx[start + i] * ne + a]];
                local[i * ne + a] = l;
                valence[l]++;
            }
        // colour: try RCB order and highest-conflict-first, keep the fewer rounds
        order.resize(E);
        std::iota(order.begin(), order.end(), 0);
        int R1 = colour_tile(order, local, ne, nl, round_of);
        std::vector<int> conflict(E, 0);
        for (int i = 0; i < E; ++i)
            for (int a = 0; a < ne; ++a) conflict[i] += valence[local[i * ne + a]];
        order2 = order;
        std::stable_sort(order2.begin(), order2.end(),
                         [&](int a, int b) { return conflict[a] > conflict[b]; });
        int R2 = colour_tile(order2, local, ne, nl, round_of2);
        if (R2 < R1) {
            R1 = R2;
            round_of.swap(round_of2);
        }
        // iterated greedy: revisit elements class by class (largest classes
        // last, then reversed); first-fit never needs more rounds than the
        // ordering it is fed, so the count can only drop.
        for (int it = 0; it < 12 && R1 <= kMaxRounds; ++it) {
            std::vector<int> size(R1, 0);
            for (int i = 0; i < E; ++i) size[round_of[i]]++;
            std::vector<int> cls(R1);
            std::iota(cls.begin(), cls.end(), 0);
            if (it % 3 == 0)
                std::stable_sort(cls.begin(), cls.end(), [&](int a, int b) { return size[a] < size[b]; });
            else if (it % 3 == 1)
                std::reverse(cls.begin(), cls.end());
            else
                std::stable_sort(cls.begin(), cls.end(), [&](int a, int b) { return size[a] > size[b]; });
            std::vector<int> rank(R1);
            for (int k = 0; k < R1; ++k) rank[cls[k]] = k;
            order2.resize(E);
            std::iota(order2.begin(), order2.end(), 0);
            std::stable_sort(order2.begin(), order2.end(),
                             [&](int a, int b) { return rank[round_of[a]] < rank[round_of[b]]; });
            int R2 = colour_tile(order2, local, ne, nl, round_of2);
            if (R2 <= R1) {
                R1 = R2;
                round_of.swap(round_of2);
            }
        }
        if (R1 > kMaxRounds) return "tile needs more than 128 rounds";
        // emit rounds
        int64_t r0 = P.n_rounds();
        P.round_elem.resize((size_t)(r0 + R1) * kRound, -1);
        P.round_nvalid.resize(r0 + R1, 0);
        P.round_conn.resize((size_t)(r0 + R1) * kRound * P.n_en_pad, 0);
        for (int i = 0; i < E; ++i) {
            int64_t r = r0 + round_of[i];
            int lane = P.round_nvalid[r]++;
            P.round_elem[r * kRound + lane] = idx[start + i];
            for (int a = 0; a < ne; ++a)
                P.round_conn[(r * kRound + lane) * P.n_en_pad + a] = (uint16_t)local[i * ne + a];
        }
        P.max_rounds = std::max(P.max_rounds, R1);
        P.max_tile_nodes = std::max(P.max_tile_nodes, nl);
        P.tile_round_ptr.push_back((int32_t)(r0 + R1));
        for (int j = 0; j < nl; ++j) {
            P.node_gid.push_back(gids[j]);
            loc[gids[j]] = -1;
        }
        P.tile_node_ptr.push_back((int64_t)P.node_gid.size());
        start = end;
    }

    // shared nodes and their slots (slots of a node in ascending tile order)
    std::vector<int32_t> sid_of(NN, -1);
    P.shared_slot_ptr.assign(1, 0);
    for (int64_t n = 0; n < NN; ++n) {
        if (tiles_of_node[n] == 0) P.orphans.push_back((int32_t)n);
        if (tiles_of_node[n] >= 2) {
            sid_of[n] = (int32_t)P.shared_gid.size();
            P.shared_gid.push_back((int32_t)n);
            P.shared_slot_ptr.push_back(P.shared_slot_ptr.back() + tiles_of_node[n]);
        }
    }
    P.slot_owner.assign(P.shared_slot_ptr.back(), -1);
    std::vector<int64_t> fill(P.shared_gid.size(), 0);
    P.node_slot.assign(P.node_gid.size(), -1);
    for (int t = 0; t < nt; ++t)
        for (int64_t j = P.tile_node_ptr[t]; j < P.tile_node_ptr[t + 1]; ++j) {
            int32_t s = sid_of[P.node_gid[j]];
            if (s < 0) continue;
            int64_t slot = P.shared_slot_ptr[s] + fill[s]++;
            if (slot > INT32_MAX) return "too many partial slots";
            P.node_slot[j] = (int32_t)slot;
            P.slot_owner[slot] = s;
        }
    return "";
}

}  // namespace fem
