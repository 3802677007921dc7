// Host-side two-level partition (see fem_plan.h).  Pure C++, no CUDA, so the
// colouring can be built and checked on a machine without a GPU.
#include "fem_plan.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>

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

// Fewest rounds a tile allows: ceil(E / 32).  The greedy colourings above
// leave most 1024-element tet tiles one round over it (33 rounds of ~31
// elements), which costs the two-elements-per-lane kernels a fifth, half-empty
// pair of rounds on one warp of every tile.  A tabu search repairs that: the
// elements of the extra rounds go to the rounds with room and the fewest
// clashes, then every step swaps a clashing element with the element of
// another round (or moves it to a round with room) that lowers the number of
// same-round element pairs sharing a node the most, and bars the reverse for
// a few steps.  Ties and the element to repair are drawn from a fixed-seed
// generator, so the plan stays a function of the mesh.  Returns false, with
// round_of untouched, when no clash-free colouring is found in max_steps.
bool tighten_rounds(int E, int ne, int nl, const std::vector<int>& local, std::vector<int>& round_of, int R,
                    uint64_t seed, int max_steps = 4000) {
    const int Rt = (E + kRound - 1) / kRound;
    if (R <= Rt || Rt <= 0) return false;
    uint64_t st = seed;
    auto next = [&]() {  // splitmix64
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<int> ro(E, -1), size(Rt, 0);
    std::vector<uint8_t> cnt((size_t)Rt * nl, 0);  // elements of round r on node n
    auto at = [&](int r, int n) -> uint8_t& { return cnt[(size_t)r * nl + n]; };
    auto put = [&](int e, int r) {
        for (int a = 0; a < ne; ++a) ++at(r, local[e * ne + a]);
        ++size[r];
        ro[e] = r;
    };
    auto take = [&](int e) {
        const int r = ro[e];
        for (int a = 0; a < ne; ++a) --at(r, local[e * ne + a]);
        --size[r];
    };
    auto seen = [&](int e, int r) {  // e's node clashes with the elements of round r
        int c = 0;
        for (int a = 0; a < ne; ++a) c += at(r, local[e * ne + a]);
        return c;
    };
    for (int e = 0; e < E; ++e)
        if (round_of[e] < Rt) put(e, round_of[e]);
    for (int e = 0; e < E; ++e) {
        if (round_of[e] < Rt) continue;
        int best = -1, bc = 1 << 30;
        for (int r = 0; r < Rt; ++r)
            if (size[r] < kRound && seen(e, r) < bc) bc = seen(e, r), best = r;
        put(e, best);  // total room is Rt * 32 >= E, so some round has room
    }
    std::vector<int> tabu((size_t)E * Rt, -1), conf(E), bad;
    for (int step = 0; step < max_steps; ++step) {
        bad.clear();
        for (int e = 0; e < E; ++e) {
            conf[e] = seen(e, ro[e]) - ne;
            if (conf[e] > 0) bad.push_back(e);
        }
        if (bad.empty()) {
            round_of = ro;
            return true;
        }
        const int e = bad[next() % bad.size()];
        const int r = ro[e];
        const int* ev = &local[e * ne];
        int best_f = -1, best_s = -1, best_d = 1 << 30;
        uint64_t best_key = 0;
        auto offer = [&](int f, int s, int d) {
            const uint64_t key = next();
            if (d < best_d || (d == best_d && key < best_key)) best_d = d, best_f = f, best_s = s, best_key = key;
        };
        for (int s = 0; s < Rt; ++s)  // moves into rounds with room
            if (s != r && size[s] < kRound && tabu[(size_t)e * Rt + s] < step) offer(-1, s, seen(e, s) - conf[e]);
        for (int f = 0; f < E; ++f) {
            const int s = ro[f];
            if (s == r || tabu[(size_t)e * Rt + s] >= step || tabu[(size_t)f * Rt + r] >= step) continue;
            const int* fv = &local[f * ne];
            int sh = 0;
            for (int a = 0; a < ne; ++a)
                for (int b = 0; b < ne; ++b) sh += ev[a] == fv[b];
            offer(f, s, (seen(e, s) - sh) + (seen(f, r) - sh) - conf[e] - conf[f]);
        }
        if (best_s < 0) continue;
        const int tenure = 7 + (int)(next() % 10);
        take(e);
        if (best_f >= 0) {
            take(best_f);
            put(best_f, r);
            tabu[(size_t)best_f * Rt + best_s] = step + tenure;
        }
        put(e, best_s);
        tabu[(size_t)e * Rt + r] = step + tenure;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Bank-conflict-free arrangement of P1 rounds.
//
// The kernels keep one nodal vector per local node in shared memory (16 B in
// 3D FP32, 8 B in 2D FP32), so a warp-wide gather of vertex slot a of a round
// touches shared-memory "bank groups" local_id mod R (R = 128 B / vector size)
// and is served one phase of R lanes at a time.  It costs one wavefront per
// phase exactly when the R lanes of the phase hit R different groups.  Three
// free choices make that happen:
//   1. the local numbering: residues mod R balanced inside every round;
//   2. which elements share a phase: each phase of R elements carries each
//      residue exactly NEN times (greedy fill, then pairwise swaps);
//   3. each element's vertex order: with every residue at most NEN times in a
//      phase, the element/residue bipartite multigraph has maximum degree NEN,
//      so by Koenig's theorem its edges split into NEN matchings -- slot s of
//      the phase takes the nodes of matching s, all in different groups.
// P1 elements accept any vertex order (their shape-function gradients are
// computed for the order chosen).
// ---------------------------------------------------------------------------

// Relabel the tile's nodes so that residue classes mod R are balanced per
// round.  Returns new_id[old_local].  Class b gets exactly the ids of [0, nl)
// congruent to b, so the result is a permutation.
std::vector<int> balanced_labels(int nl, int E, int ne, const std::vector<int>& local,
                                 const std::vector<int>& round_of, int R_rounds, int R) {
    std::vector<std::vector<int>> node_rounds(nl);
    for (int i = 0; i < E; ++i)
        for (int a = 0; a < ne; ++a) node_rounds[local[i * ne + a]].push_back(round_of[i]);
    std::vector<int> order(nl);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return node_rounds[a].size() > node_rounds[b].size();
    });
    std::vector<int> cap(R), used(R, 0), res(nl, 0);
    for (int b = 0; b < R; ++b) cap[b] = (nl - b + R - 1) / R;
    std::vector<int> cnt((size_t)R_rounds * R, 0);
    for (int n : order) {
        int best = -1;
        long best_cost = 0;
        for (int b = 0; b < R; ++b) {
            if (used[b] >= cap[b]) continue;
            long c = 0;
            for (int r : node_rounds[n]) {
                const int x = cnt[(size_t)r * R + b];
                c += (long)x * x;  // convex: spreads residues within each round
            }
            if (best < 0 || c < best_cost || (c == best_cost && used[b] < used[best])) {
                best = b;
                best_cost = c;
            }
        }
        res[n] = best;
        used[best]++;
        for (int r : node_rounds[n]) cnt[(size_t)r * R + best]++;
    }
    // local search: swap the classes of two nodes when that lowers the number
    // of residues above the round's even share (deterministic xorshift draws)
    std::vector<int> target(R_rounds, 0);
    for (int r = 0; r < R_rounds; ++r) {
        int tot = 0;
        for (int b = 0; b < R; ++b) tot += cnt[(size_t)r * R + b];
        target[r] = (tot + R - 1) / R;
    }
    auto over = [&](int r, int b, int delta) {
        const int x = cnt[(size_t)r * R + b];
        return std::max(0, x + delta - target[r]) - std::max(0, x - target[r]);
    };
    uint64_t st = 0x9E3779B97F4A7C15ull ^ (uint64_t)nl * 0x2545F4914F6CDD1Dull;
    auto rnd = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return st;
    };
    const int iters = 40 * nl;
    for (int k = 0; k < iters && nl > 1; ++k) {
        const int i = (int)(rnd() % nl), j = (int)(rnd() % nl);
        const int bi = res[i], bj = res[j];
        if (bi == bj) continue;
        int d = 0;
        for (int r : node_rounds[i]) d += over(r, bi, -1) + over(r, bj, +1);
        for (int r : node_rounds[i]) {
            cnt[(size_t)r * R + bi]--;
            cnt[(size_t)r * R + bj]++;
        }
        for (int r : node_rounds[j]) d += over(r, bj, -1) + over(r, bi, +1);
        if (d < 0) {
            for (int r : node_rounds[j]) {
                cnt[(size_t)r * R + bj]--;
                cnt[(size_t)r * R + bi]++;
            }
            res[i] = bj;
            res[j] = bi;
        } else {
            for (int r : node_rounds[i]) {
                cnt[(size_t)r * R + bi]++;
                cnt[(size_t)r * R + bj]--;
            }
        }
    }
    std::vector<int> next(R, 0), new_id(nl);
    for (int n = 0; n < nl; ++n) new_id[n] = res[n] + R * next[res[n]]++;
    return new_id;
}

// Colour the edges of a bipartite multigraph (left: elements of one phase,
// right: residues) with `ne` colours so that no two edges of one colour share
// a vertex.  Edges beyond `ne` at a residue cannot all be placed; they are set
// aside, the rest (maximum degree ne on both sides) is coloured properly by
// alternating-path recolouring (Koenig), and each set-aside edge then takes a
// colour still free at its element.  Every element ends with distinct colours.
void colour_phase(int n_el, int ne, int R, const std::vector<int>& res_of_edge /* [n_el*ne] */,
                  std::vector<int>& slot_of_edge) {
    const int NE = n_el * ne;
    slot_of_edge.assign(NE, -1);
    std::vector<int> at_l((size_t)n_el * ne, -1), at_r((size_t)R * ne, -1);  // edge holding a colour
    std::vector<int> deg(R, 0);
    std::vector<char> extra(NE, 0);
    for (int e = 0; e < NE; ++e)
        if (++deg[res_of_edge[e]] > ne) extra[e] = 1;
    auto left = [&](int e) { return e / ne; };
    for (int e = 0; e < NE; ++e) {
        if (extra[e]) continue;
        const int l = left(e), r = res_of_edge[e];
        int alpha = -1, beta = -1;
        for (int c = 0; c < ne && alpha < 0; ++c)
            if (at_l[(size_t)l * ne + c] < 0) alpha = c;
        for (int c = 0; c < ne && beta < 0; ++c)
            if (at_r[(size_t)r * ne + c] < 0) beta = c;
        if (at_r[(size_t)r * ne + alpha] >= 0) {
            // swap alpha/beta along the path that starts at r with colour alpha;
            // in a bipartite graph it cannot reach l
            std::vector<int> path;
            int cur_r = r, cur_l = -1, c = alpha;
            bool on_right = true;
            for (int guard = 0; guard <= NE; ++guard) {
                const int f = on_right ? at_r[(size_t)cur_r * ne + c] : at_l[(size_t)cur_l * ne + c];
                if (f < 0) break;
                path.push_back(f);
                if (on_right)
                    cur_l = left(f);
                else
                    cur_r = res_of_edge[f];
                on_right = !on_right;
                c = (c == alpha) ? beta : alpha;
            }
            for (int f : path) {
                at_l[(size_t)left(f) * ne + slot_of_edge[f]] = -1;
                at_r[(size_t)res_of_edge[f] * ne + slot_of_edge[f]] = -1;
            }
            for (int f : path) {
                const int cf = slot_of_edge[f] == alpha ? beta : alpha;
                slot_of_edge[f] = cf;
                at_l[(size_t)left(f) * ne + cf] = f;
                at_r[(size_t)res_of_edge[f] * ne + cf] = f;
            }
        }
        slot_of_edge[e] = alpha;
        at_l[(size_t)l * ne + alpha] = e;
        at_r[(size_t)r * ne + alpha] = e;
    }
    for (int e = 0; e < NE; ++e) {
        if (!extra[e]) continue;
        const int l = left(e);
        for (int c = 0; c < ne; ++c)
            if (at_l[(size_t)l * ne + c] < 0) {
                slot_of_edge[e] = c;
                at_l[(size_t)l * ne + c] = e;
                break;
            }
    }
}

// Order the elements of one round into lanes and their vertices into slots.
// elems: tile-local element indices; lid: new local ids per element vertex.
// Output: lane order and, per lane, the vertex permutation (slot -> vertex).
void arrange_round(const std::vector<int>& elems, int ne, int R, const std::vector<int>& lid,
                   std::vector<int>& lane_elem, std::vector<int>& perm) {
    const int n = (int)elems.size();
    const int G = R;  // lanes per phase
    const int n_ph = (n + G - 1) / G;
    auto resv = [&](int k, int a) { return lid[elems[k] * ne + a] % R; };
    // greedy fill of phases (sizes G, G, ..., remainder) from several element
    // orders, each followed by pairwise swaps; keep the lowest excess
    std::vector<int> cap(n_ph, G);
    cap[n_ph - 1] = n - G * (n_ph - 1);
    std::vector<int> ph_of(n), best_ph(n), cnt((size_t)n_ph * R, 0), size(n_ph, 0);
    auto cost_add = [&](int q, int k, int sign) {
        long c = 0;
        for (int a = 0; a < ne; ++a) {
            int& x = cnt[(size_t)q * R + resv(k, a)];
            if (sign > 0) {
                c += (x >= ne) ? 1 : 0;
                x++;
            } else {
                x--;
                c -= (x >= ne) ? 1 : 0;
            }
        }
        return c;
    };
    long best_total = -1;
    uint64_t st = 0xD1B54A32D192ED03ull ^ (uint64_t)(n * 131 + lid[elems[0] * ne]);
    std::vector<int> order(n);
    for (int attempt = 0; attempt < 4; ++attempt) {
        std::iota(order.begin(), order.end(), 0);
        if (attempt > 0)
            for (int k = n - 1; k > 0; --k) {  // Fisher-Yates with xorshift draws
                st ^= st << 13;
                st ^= st >> 7;
                st ^= st << 17;
                std::swap(order[k], order[(int)(st % (uint64_t)(k + 1))]);
            }
        std::fill(cnt.begin(), cnt.end(), 0);
        std::fill(size.begin(), size.end(), 0);
        long total = 0;
        for (int k : order) {
            int best = -1;
            long bc = 0;
            for (int q = 0; q < n_ph; ++q) {
                if (size[q] >= cap[q]) continue;
                const long c = cost_add(q, k, +1);
                cost_add(q, k, -1);
                if (best < 0 || c < bc) {
                    best = q;
                    bc = c;
                }
            }
            ph_of[k] = best;
            size[best]++;
            total += cost_add(best, k, +1);
        }
        for (int pass = 0; pass < 4; ++pass) {
            bool improved = false;
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) {
                    const int qi = ph_of[i], qj = ph_of[j];
                    if (qi == qj) continue;
                    long d = cost_add(qi, i, -1) + cost_add(qj, j, -1);
                    d += cost_add(qi, j, +1) + cost_add(qj, i, +1);
                    if (d < 0) {
                        ph_of[i] = qj;
                        ph_of[j] = qi;
                        total += d;
                        improved = true;
                    } else {
                        cost_add(qi, j, -1);
                        cost_add(qj, i, -1);
                        cost_add(qi, i, +1);
                        cost_add(qj, j, +1);
                    }
                }
            if (!improved) break;
        }
        if (best_total < 0 || total < best_total) {
            best_total = total;
            best_ph = ph_of;
        }
        if (best_total == 0) break;
    }
    ph_of = best_ph;
    // lanes: phase by phase; vertex slots by edge colouring inside each phase
    lane_elem.clear();
    perm.assign((size_t)n * ne, 0);
    for (int q = 0; q < n_ph; ++q) {
        std::vector<int> members;
        for (int k = 0; k < n; ++k)
            if (ph_of[k] == q) members.push_back(k);
        std::vector<int> res_e(members.size() * ne), slot;
        for (size_t m = 0; m < members.size(); ++m)
            for (int a = 0; a < ne; ++a) res_e[m * ne + a] = resv(members[m], a);
        colour_phase((int)members.size(), ne, R, res_e, slot);
        for (size_t m = 0; m < members.size(); ++m) {
            const int lane = (int)lane_elem.size();
            lane_elem.push_back(members[m]);
            // vertex a goes to slot slot[m*ne+a]; keep the input order should
            // the colours of an element not form a permutation
            int seen = 0;
            for (int a = 0; a < ne; ++a) {
                const int sl = slot[m * ne + a];
                if (sl >= 0 && sl < ne) seen |= 1 << sl;
            }
            for (int a = 0; a < ne; ++a)
                perm[(size_t)lane * ne + (seen == (1 << ne) - 1 ? slot[m * ne + a] : a)] = a;
        }
    }
}

// Everything one tile needs, built independently of the other tiles.
struct TileOut {
    std::string err;
    std::vector<int32_t> gid;        // [nl] global id of each local node (final numbering)
    std::vector<int32_t> elem;       // [R*32] element per (round, lane) or -1
    std::vector<uint8_t> nvalid;     // [R]
    std::vector<uint16_t> conn;      // [R*32*pad] local ids in slot order
    int rounds = 0;
};

void build_tile(const MeshInput& in, const int32_t* elems, int E, int pad, TileOut& out) {
    const int ne = in.n_en;
    // local node numbering: ascending global id
    std::vector<int32_t> gids;
    gids.reserve((size_t)E * ne);
    for (int i = 0; i < E; ++i)
        for (int a = 0; a < ne; ++a) gids.push_back(in.conn[(int64_t)elems[i] * ne + a]);
    std::sort(gids.begin(), gids.end());
    gids.erase(std::unique(gids.begin(), gids.end()), gids.end());
    const int nl = (int)gids.size();
    if (nl > 65535) {
        out.err = "tile has more than 65535 nodes";
        return;
    }
    std::vector<int> local((size_t)E * ne), valence(nl, 0);
    for (int i = 0; i < E; ++i)
        for (int a = 0; a < ne; ++a) {
            const int32_t g = in.conn[(int64_t)elems[i] * ne + a];
            const int l = (int)(std::lower_bound(gids.begin(), gids.end(), g) - gids.begin());
            local[i * ne + a] = l;
            valence[l]++;
        }
    // colour: try the RCB order and highest-conflict-first, keep the fewer rounds
    std::vector<int> order(E), order2, round_of, round_of2;
    std::iota(order.begin(), order.end(), 0);
    int R1 = colour_tile(order, local, ne, nl, round_of);
    std::vector<int> conflict(E, 0);
    for (int i = 0; i < E; ++i)
        for (int a = 0; a < ne; ++a) conflict[i] += valence[local[i * ne + a]];
    order2 = order;
    std::stable_sort(order2.begin(), order2.end(), [&](int a, int b) { return conflict[a] > conflict[b]; });
    int R2 = colour_tile(order2, local, ne, nl, round_of2);
    if (R2 < R1) {
        R1 = R2;
        round_of.swap(round_of2);
    }
    // classes first: an uncapacitated first-fit colouring, its classes
    // visited one after the other, each split into rounds by the capacitated
    // first-fit.  The uncapacitated pass visits the elements in RCB order and
    // in the lexicographic orders of their centroids (on structured grids the
    // latter give the cell parities, 8 classes for Q1, which fill every round)
    {
        std::vector<double> cen((size_t)E * in.dim, 0.0);
        for (int i = 0; i < E; ++i)
            for (int a = 0; a < ne; ++a)
                for (int c = 0; c < in.dim; ++c)
                    cen[(size_t)i * in.dim + c] += in.X[(int64_t)in.conn[(int64_t)elems[i] * ne + a] * in.dim + c];
        for (int variant = 0; variant < 3; ++variant) {
            std::vector<int> visit(E);
            std::iota(visit.begin(), visit.end(), 0);
            if (variant > 0)
                std::stable_sort(visit.begin(), visit.end(), [&](int a, int b) {
                    for (int k = 0; k < in.dim; ++k) {
                        const int c = variant == 1 ? in.dim - 1 - k : k;  // slowest axis first
                        const double x = cen[(size_t)a * in.dim + c], y = cen[(size_t)b * in.dim + c];
                        if (x != y) return x < y;
                    }
                    return false;
                });
            std::vector<u128> used(nl, 0);
            std::vector<int> cls(E);
            for (int i : visit) {
                u128 m = 0;
                for (int a = 0; a < ne; ++a) m |= used[local[i * ne + a]];
                const int c = lowest_zero(m);
                cls[i] = c;
                if (c < 128)
                    for (int a = 0; a < ne; ++a) used[local[i * ne + a]] |= (u128)1 << c;
            }
            order2 = visit;
            std::stable_sort(order2.begin(), order2.end(), [&](int a, int b) { return cls[a] < cls[b]; });
            R2 = colour_tile(order2, local, ne, nl, round_of2);
            if (R2 < R1) {
                R1 = R2;
                round_of.swap(round_of2);
            }
        }
    }
    // iterated greedy: revisit elements class by class (largest classes last,
    // then reversed); first-fit never needs more rounds than the ordering it
    // is fed, so the count can only drop.
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
        R2 = colour_tile(order2, local, ne, nl, round_of2);
        if (R2 <= R1) {
            R1 = R2;
            round_of.swap(round_of2);
        }
    }
    if (R1 > kMaxRounds) {
        out.err = "tile needs more than 128 rounds";
        return;
    }
    // a round holds at most one element of each node, so a tile needs at
    // least as many rounds as its busiest node has elements: the repair is
    // tried only where the floor allows that
    const int floor_rounds = (E + kRound - 1) / kRound;
    const int max_valence = nl > 0 ? *std::max_element(valence.begin(), valence.end()) : 0;
    if (max_valence <= floor_rounds &&
        tighten_rounds(E, ne, nl, local, round_of, R1, 0x5EEDull ^ (uint64_t)(uint32_t)elems[0]))
        R1 = floor_rounds;
    // P1 tiles are relabelled and arranged so that the warp-wide
    // shared-memory gathers are free of bank conflicts
    const bool arrange = in.arrange && in.elem_type != 2;
    const int Rq = in.dim == 2 ? 16 : 8;
    std::vector<int> new_id(nl);
    std::iota(new_id.begin(), new_id.end(), 0);
    if (arrange) new_id = balanced_labels(nl, E, ne, local, round_of, R1, Rq);
    std::vector<int> lid((size_t)E * ne);
    for (int i = 0; i < E * ne; ++i) lid[i] = new_id[local[i]];
    out.rounds = R1;
    out.elem.assign((size_t)R1 * kRound, -1);
    out.nvalid.assign(R1, 0);
    out.conn.assign((size_t)R1 * kRound * pad, kNoNode);  // empty lanes hold kNoNode
    std::vector<std::vector<int>> members(R1);
    for (int i = 0; i < E; ++i) members[round_of[i]].push_back(i);
    std::vector<int> lane_elem, perm;
    for (int r = 0; r < R1; ++r) {
        const std::vector<int>& mem = members[r];
        if (arrange) {
            arrange_round(mem, ne, Rq, lid, lane_elem, perm);
        } else {
            lane_elem.resize(mem.size());
            std::iota(lane_elem.begin(), lane_elem.end(), 0);
            perm.resize(mem.size() * ne);
            for (size_t k = 0; k < mem.size(); ++k)
                for (int a = 0; a < ne; ++a) perm[k * ne + a] = a;
        }
        out.nvalid[r] = (uint8_t)mem.size();
        for (size_t lane = 0; lane < mem.size(); ++lane) {
            const int i = mem[lane_elem[lane]];
            out.elem[(size_t)r * kRound + lane] = elems[i];
            for (int sl = 0; sl < ne; ++sl)
                out.conn[((size_t)r * kRound + lane) * pad + sl] = (uint16_t)lid[i * ne + perm[lane * ne + sl]];
        }
    }
    out.gid.assign(nl, 0);
    for (int j = 0; j < nl; ++j) out.gid[new_id[j]] = gids[j];
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

    // tiles are independent: build them on the host's cores, assemble in order
    std::vector<TileOut> tiles(nt);
    std::vector<int64_t> first(nt);
    for (int t = 0; t < nt; ++t) first[t] = t ? leaves[t - 1] : 0;
    const int nthreads = std::max(1, std::min<int>(nt, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int t = next++; t < nt; t = next++)
            build_tile(in, idx.data() + first[t], (int)(leaves[t] - first[t]), P.n_en_pad, tiles[t]);
    };
    std::vector<std::thread> pool;
    for (int k = 1; k < nthreads; ++k) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();

    std::vector<int32_t> tiles_of_node(NN, 0);
    P.tile_round_ptr.assign(1, 0);
    P.tile_node_ptr.assign(1, 0);
    for (int t = 0; t < nt; ++t) {
        TileOut& o = tiles[t];
        if (!o.err.empty()) return o.err;
        P.round_elem.insert(P.round_elem.end(), o.elem.begin(), o.elem.end());
        P.round_nvalid.insert(P.round_nvalid.end(), o.nvalid.begin(), o.nvalid.end());
        P.round_conn.insert(P.round_conn.end(), o.conn.begin(), o.conn.end());
        P.max_rounds = std::max(P.max_rounds, o.rounds);
        P.max_tile_nodes = std::max(P.max_tile_nodes, (int)o.gid.size());
        P.tile_round_ptr.push_back(P.tile_round_ptr.back() + o.rounds);
        for (int32_t g : o.gid) tiles_of_node[g]++;
        P.node_gid.insert(P.node_gid.end(), o.gid.begin(), o.gid.end());
        // pad the tile's node list to kNodeAlign entries (bulk-copyable)
        while (P.node_gid.size() % kNodeAlign) P.node_gid.push_back(-1);
        P.tile_node_ptr.push_back((int64_t)P.node_gid.size());
        o = TileOut();  // release the tile's buffers
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
            if (P.node_gid[j] < 0) continue;  // padding
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
