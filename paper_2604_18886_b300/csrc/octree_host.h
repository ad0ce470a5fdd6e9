// Host-side octree construction and multigrid tables for libocg.
//
// Layout used by every kernel (see kernels.cuh):
//  * Multigrid levels m = D (finest) .. mc (coarsest).  Level m >= 0 holds every cell
//    of depth m (leaves and inner); level m < 0 is the uniform coarsening of the root
//    grid by 2^-m.  The coarsest grid is padded to an even size with inactive cells.
//  * Cells of a level are stored in octets: the 8 children of one cell of the next
//    coarser grid, slot s = dx + 2 dy + 4 dz.  On the adaptive levels (m >= 1) octets are
//    sorted by the Morton key of their parent; on the uniform levels (m <= 0) they are in
//    lexicographic order of the parent, so neighbouring octets are found arithmetically.
//  * Levels are concatenated in the order 0, 1, ..., D, -1, -2, ..., mc; cells of the
//    tree levels 0..D form the prefix [0, n_tree) that the Krylov vectors cover.
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <utility>
#include <string>
#include <vector>

#include "../../include/ocg.h"

namespace ocg {

// Allocator whose element construction without arguments leaves trivially constructible
// values uninitialised, for large work arrays that a parallel pass fills completely: a
// value-initialising resize would zero them on one thread first.
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept {
        ::new ((void*)p) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};


struct LevelMeta {
    int m = 0;        // level index (depth for m >= 0)
    int N = 0;        // cells per axis of the level grid
    int Np = 0;       // padded size (N rounded up to even at the coarsest level)
    int ni = 0;       // uniform levels (m <= 0): octets per axis, octets in lexicographic
                      // order o = I + ni (J + ni K); 0 for the adaptive levels m >= 1
    int64_t off = 0;  // first global cell
    int64_t ncell = 0;
    int64_t oct_off = 0;  // first global octet (= off / 8)
    int64_t noct = 0;
    double h = 0.0;   // cell size for m >= 0
};

struct HostTree {
    ocg_octree_desc desc{};
    int n0 = 0, D = 0, mc = 0;
    std::vector<LevelMeta> lv;          // indexed by m - mc
    std::vector<int> order;             // storage order of levels (values m)
    int64_t ncell = 0, noct = 0, ntree = 0, nleaf = 0, nt = 0, nface = 0;

    // octet parent keys per level (sorted Morton keys of the parent coordinates)
    std::vector<std::vector<uint64_t>> okeys;  // indexed by m - mc

    // refinement predicate flags per depth d < D before the 2:1 closure (dense,
    // lexicographic), kept for rebuild_host_tree
    std::vector<std::vector<uint8_t>> pred;

    // global tables
    std::vector<int32_t> nbr;        // [6][noct]: level-local octet, -1 wall, -2-K T face
                                     //   (K = global cell of the coarser leaf)
    std::vector<int32_t> oct_parent; // [noct]: global parent cell, -1 at the coarsest level
    std::vector<int32_t> child_oct;  // [ncell]: global octet of the children, -1 if none
    std::vector<int32_t> trec;       // [noct]: T record of the octet, -1 if it has no T face
    std::vector<int32_t> t_oct;      // [nt]: global octet owning the record
    std::vector<int32_t> leaf_cell;  // [nleaf]: canonical rank -> global cell
    std::vector<int64_t> leaf_first; // [D+2]: first canonical rank of each depth
    std::vector<int32_t> cell_rank;  // [ncell]: global cell -> canonical rank or -1
    std::vector<uint8_t> cell_flags; // [ncell]: bit0 leaf, bit1 active-able (not padding)
    std::vector<int8_t> cell_level;  // [ncell]

    // canonical leaves
    std::vector<int32_t> leaf_depth, leaf_i, leaf_j, leaf_k;
    // canonical faces (the + cell's coordinates follow from the leaves: face_plus_cell)
    // (uninitialised on resize: the parallel merge writes every entry, and zero-filling
    // ~19 bytes per face first cost more than the merge)
    std::vector<int8_t, NoInitAlloc<int8_t>> f_axis, f_depth;
    std::vector<int32_t, NoInitAlloc<int32_t>> f_minus, f_plus;  // canonical leaf ranks of the two sides
    std::vector<int64_t, NoInitAlloc<int64_t>> f_slot;     // destination of -beta*h (see setup kernel)
    std::vector<uint8_t, NoInitAlloc<uint8_t>> f_kind;     // 0: c_{a-} of a cell, 1: T record + face weight

    const LevelMeta& L(int m) const { return lv[m - mc]; }
    LevelMeta& L(int m) { return lv[m - mc]; }
    int64_t cell_index(int m, int64_t i, int64_t j, int64_t k) const;  // -1 if absent
    void cell_coords(int m, int64_t g, int64_t& i, int64_t& j, int64_t& k) const;
};

// Builds everything; throws std::runtime_error with a message on invalid input.
void build_host_tree(const ocg_octree_desc& desc, HostTree& T);

// Builds the octree of desc from prev, evaluating the refinement predicate only for the
// cells that meet box = (lox, loy, loz, hix, hiy, hiz) or whose parent's flag changed.  When
// the predicate of desc equals that of prev.desc on every cell that does not meet the box,
// the result equals build_host_tree(desc) exactly.  n0, max_depth and refine must match.
void rebuild_host_tree(const HostTree& prev, const ocg_octree_desc& desc, const double box[6], HostTree& T);

// Integer coordinates (at the face's depth) of the cell on the + side of canonical face f;
// for a T sub-face whose fine leaf is on the - side that cell is virtual.
void face_plus_cell(const HostTree& T, int64_t f, int32_t& i, int32_t& j, int32_t& k);

// Neighbour code of leaf r in direction dir (x-, x+, y-, y+, z-, z+): kind 0 wall, 1 same-depth
// leaf, 2 coarser leaf, 3 refined neighbour; rank = canonical rank for kinds 1 and 2, else -1.
void leaf_neighbour(const HostTree& T, int64_t r, int dir, int8_t& kind, int64_t& rank);

// Topology of A^T - A of the composite leaf operator.  Only T-junctions make A non-symmetric:
// a T sub-face f of the fine leaf i against the coarser leaf K contributes
// (w_f/2) [(a_P - e_K)(e_i - e_K)^T - (e_i - e_K)(a_P - e_K)^T], a_P the averaging weights of
// the leaves under i's parent P (1/8 per level; every tree cell is taken as active).  The
// correction is applied matrix-free (kernels k_tfine, k_tcoarse, k_tdesc) from
//   tcoarse: the coarse leaves K (global cells, sorted, unique);
//   tdesc:   every T octet and every octet below one (global octets, each once), whose
//            leaves receive the a_P terms.
struct AdjointTopology {
    std::vector<int32_t> tcoarse, tdesc;
};
void build_adjoint_topology(const HostTree& T, AdjointTopology& out);

// Geometry of OCG_REFINE_SDF_BAND descriptions: the solids' signed distance (positive in
// fluid), and the clamped FP32 fluid fraction of the - face along `axis` of cell (i, j, k)
// of level m (cell size 1 / (n0 2^m)): the face split into two triangles along its
// (0,0)-(1,1) diagonal in the two other axes (increasing order), phi linear on each from
// its corner values, the positive area exact; max(1e-3, min(1, f)) rounded to FP32.
double solid_sdf(const ocg_octree_desc& d, double x, double y, double z);
float face_beta_geometric(const ocg_octree_desc& d, int m, int axis, int64_t i, int64_t j, int64_t k);

uint64_t morton3(uint64_t i, uint64_t j, uint64_t k);
void demorton3(uint64_t key, uint64_t& i, uint64_t& j, uint64_t& k);

}  // namespace ocg
