// Host-side mesh plan: the two-level partition of the element set that makes
// the device scatter deterministic and free of value atomics.
//
// Level 1 (tiles): recursive coordinate bisection of element centroids into
//   spatially compact tiles of at most `tile_elems` elements.  One CTA owns a
//   tile; the tile's nodes get a local u16 numbering and live in shared
//   memory while the CTA runs.
// Level 2 (rounds): inside a tile, elements are coloured into rounds of at
//   most 32 elements that share no node (first-fit colouring with capacity
//   32, highest-conflict elements first).  A warp processes one round at a
//   time, one element per lane, so no two lanes ever update the same node.
// Between tiles: a node touched by one tile is written by that tile alone;
//   a node touched by several tiles ("shared") receives one partial per
//   tile in a fixed slot, and the slots are summed in tile order.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fem {

constexpr int kRound = 32;       // elements per round (one per lane)
constexpr int kMaxRounds = 128;  // per tile (bit masks in the colourer)
constexpr int kNodeAlign = 16;   // tile node lists are padded to this many entries
constexpr uint16_t kNoNode = 0xFFFF;  // local id of an empty lane in a round

struct MeshInput {
    int elem_type = 1;  // 0 tri3, 1 tet4, 2 hex8
    int dim = 3, n_en = 4;
    int64_t n_nodes = 0, n_el = 0;
    const double* X = nullptr;
    const int32_t* conn = nullptr;
    int tile_elems = 0;
    bool arrange = true;  // bank-conflict-free lane / vertex arrangement (P1)
};

struct Plan {
    int dim = 0, n_en = 0, n_en_pad = 0, elem_type = 0;
    int64_t n_nodes = 0, n_el = 0;
    int tile_elems = 0;
    // tiles
    std::vector<int32_t> tile_round_ptr;  // [n_tiles+1]
    std::vector<int64_t> tile_node_ptr;   // [n_tiles+1], multiples of kNodeAlign
    std::vector<int32_t> node_gid;        // [n_local] global node id, -1 = padding
    std::vector<int32_t> node_slot;       // [n_local] -1: private or padding, else partial slot
    // rounds
    std::vector<int32_t> round_elem;      // [n_rounds*32] element id or -1
    std::vector<uint8_t> round_nvalid;    // [n_rounds]
    std::vector<uint16_t> round_conn;     // [n_rounds*32*n_en_pad] local node ids, in the
                                          // vertex order the kernels use (P1: may differ
                                          // from the input order; see round_elem)
    // shared nodes
    std::vector<int32_t> shared_gid;      // [n_shared]
    std::vector<int64_t> shared_slot_ptr; // [n_shared+1]
    std::vector<int32_t> slot_owner;      // [n_slots] shared id of the slot
    std::vector<int32_t> orphans;         // nodes touched by no element
    int max_tile_nodes = 0;
    int max_rounds = 0;

    int n_tiles() const { return (int)tile_round_ptr.size() - 1; }
    int64_t n_rounds() const { return (int64_t)round_nvalid.size(); }
    int64_t n_slots() const { return (int64_t)slot_owner.size(); }
};

// Build the plan.  Returns "" on success, else an error message.
std::string build_plan(const MeshInput& in, Plan& plan);

}  // namespace fem
