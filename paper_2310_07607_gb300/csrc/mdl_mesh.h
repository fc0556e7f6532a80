// mdl_mesh.h -- host-side checks of a caller-supplied forest of quad/octree leaves (Sec. 2.2).
//
// Leaves are (level, integer cell coordinates on the level grid), ordered by
// (root id, Morton key of the lower corner on the finest grid).  Used to sort and
// validate meshes given to mdl_upload_mesh (tiling, 2:1 face balance); the device
// builds its own tables and adapts the forest itself.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace mdl {

struct Leaf {
    int32_t level;
    int32_t c[3];
};

// Per-element face record kinds.
enum FaceKind { F_BOUNDARY = 0, F_SAME = 1, F_COARSER = 2, F_FINER = 3 };

struct Mesh {
    int dim = 2;
    int L = 0;                 // max refinement depth
    int base[3] = {1, 1, 1};
    int64_t fine[3] = {1, 1, 1};
    std::vector<Leaf> leaves;
    std::vector<uint64_t> keys;       // sort key of each leaf: root id, Morton index of its lower corner
    // face table, 2*dim faces per leaf
    std::vector<int8_t> kind;         // FaceKind
    std::vector<int8_t> pos;          // tangential position bits on a coarser face
    std::vector<int32_t> nbr;         // conforming/coarser: neighbour; finer: first index into hang
    std::vector<int32_t> hang;        // finer neighbours, 2^(dim-1) per hanging face
    std::vector<uint16_t> cls;        // per leaf: face configuration code sum_f kind_f 4^f (CFL class, with level)

    int nfaces() const { return 2 * dim; }
    int nsub() const { return 1 << (dim - 1); }
    int64_t n() const { return (int64_t)leaves.size(); }

    void init(int dim_, const int* base_, int L_);          // base grid of roots
    void init_params(int dim_, const int* base_, int L_);   // sizes only, no leaves
    uint64_t key(const Leaf& lf) const;
    int64_t root_id(const Leaf& lf) const;
    // Replace leaves (sorted internally); returns false + message if not a balanced tiling.
    bool set_leaves(std::vector<Leaf> lv, std::string* err);
    // Check the tiling and rebuild the face tables from `leaves` and `keys`.
    bool rebuild(std::string* err);
    // Key of the finest cell at fc, and the leaf that holds it (leaves must tile the slab).
    uint64_t cell_key(const int64_t* fc) const;
    int32_t leaf_of(const int64_t* fc) const;
    // Neighbour of leaf i across face (axis, side): kind, and data (neighbour index or
    // subface leaf list).
    int neighbour(int64_t i, int axis, int side, int32_t* out, int* posbits) const;
};

}  // namespace mdl
