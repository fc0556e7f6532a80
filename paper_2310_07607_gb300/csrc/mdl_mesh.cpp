// mdl_mesh.cpp -- host-side ordering and validation of a forest of leaves.
#include "mdl_mesh.h"

#include <algorithm>
#include <numeric>

namespace mdl {

void Mesh::init_params(int dim_, const int* base_, int L_) {
    dim = dim_;
    L = L_;
    for (int k = 0; k < 3; ++k) base[k] = (k < dim) ? base_[k] : 1;
    for (int k = 0; k < 3; ++k) fine[k] = (int64_t)base[k] << ((k < dim) ? L : 0);
}

void Mesh::init(int dim_, const int* base_, int L_) {
    init_params(dim_, base_, L_);
    leaves.clear();
    for (int z = 0; z < base[2]; ++z)
        for (int y = 0; y < base[1]; ++y)
            for (int x = 0; x < base[0]; ++x) leaves.push_back(Leaf{0, {x, y, z}});
    keys.clear();
    std::string e;
    set_leaves(leaves, &e);
}

int64_t Mesh::root_id(const Leaf& lf) const {
    const int l = lf.level;
    int64_t r[3];
    for (int k = 0; k < 3; ++k) r[k] = (k < dim) ? (lf.c[k] >> l) : 0;
    return r[0] + (int64_t)base[0] * (r[1] + (int64_t)base[1] * r[2]);
}

uint64_t Mesh::key(const Leaf& lf) const {
    const int l = lf.level;
    uint64_t loc[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        const int64_t r = lf.c[k] >> l;
        loc[k] = (uint64_t)(lf.c[k] - (r << l)) << (L - l);
    }
    uint64_t m = 0;
    for (int bit = 0; bit < L; ++bit)
        for (int k = 0; k < dim; ++k) m |= ((loc[k] >> bit) & 1ull) << (bit * dim + k);
    return ((uint64_t)root_id(lf) << (dim * L)) | m;
}

bool Mesh::set_leaves(std::vector<Leaf> lv, std::string* err) {
    std::vector<uint64_t> kk(lv.size());
    for (size_t i = 0; i < lv.size(); ++i) kk[i] = key(lv[i]);
    std::vector<int64_t> idx(lv.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return kk[a] < kk[b]; });
    leaves.resize(lv.size());
    keys.resize(lv.size());
    for (size_t i = 0; i < lv.size(); ++i) {
        leaves[i] = lv[idx[i]];
        keys[i] = kk[idx[i]];
    }
    return rebuild(err);
}

uint64_t Mesh::cell_key(const int64_t* fc) const {
    uint64_t loc[3] = {0, 0, 0};
    int64_t r[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        r[k] = fc[k] >> L;
        loc[k] = (uint64_t)(fc[k] - (r[k] << L));
    }
    uint64_t m = 0;
    for (int bit = 0; bit < L; ++bit)
        for (int k = 0; k < dim; ++k) m |= ((loc[k] >> bit) & 1ull) << (bit * dim + k);
    const uint64_t rid = (uint64_t)(r[0] + (int64_t)base[0] * (r[1] + (int64_t)base[1] * r[2]));
    return (rid << (dim * L)) | m;
}

int32_t Mesh::leaf_of(const int64_t* fc) const {
    const uint64_t k = cell_key(fc);
    return (int32_t)(std::upper_bound(keys.begin(), keys.end(), k) - keys.begin()) - 1;
}

bool Mesh::rebuild(std::string* err) {
    // The leaves, sorted by key, tile the slab exactly when each one starts where the one
    // before it ends (a leaf of level l spans 2^(d (L - l)) consecutive finest-cell keys)
    // and together they span every root.
    for (int64_t i = 0; i < n(); ++i) {
        const Leaf& lf = leaves[i];
        if (lf.level < 0 || lf.level > L) {
            if (err) *err = "leaf level out of range";
            return false;
        }
        for (int k = 0; k < dim; ++k)
            if (lf.c[k] < 0 || lf.c[k] >= ((int64_t)base[k] << lf.level)) {
                if (err) *err = "leaf outside the slab";
                return false;
            }
    }
    uint64_t next = 0;
    for (int64_t i = 0; i < n(); ++i) {
        const Leaf& lf = leaves[i];
        if (keys[i] < next) {
            if (err) *err = "leaves overlap";
            return false;
        }
        if (keys[i] > next) {
            if (err) *err = "leaves do not cover the slab";
            return false;
        }
        next = keys[i] + (1ull << (dim * (L - lf.level)));
    }
    int64_t nroots = 1;
    for (int k = 0; k < dim; ++k) nroots *= base[k];
    if (next != ((uint64_t)nroots << (dim * L))) {
        if (err) *err = "leaves do not cover the slab";
        return false;
    }
    const int NF = nfaces(), NS = nsub();
    kind.assign(n() * NF, F_BOUNDARY);
    pos.assign(n() * NF, 0);
    nbr.assign(n() * NF, -1);
    hang.clear();
    cls.assign(n(), 0);
    int32_t sub[4];
    for (int64_t i = 0; i < n(); ++i) {
        uint16_t code = 0;
        for (int f = 0; f < NF; ++f) {
            const int axis = f / 2, side = (f & 1) ? 1 : -1;
            int pb = 0;
            const int kd = neighbour(i, axis, side, sub, &pb);
            if (kd < 0) {
                if (err) *err = "mesh is not 2:1 face balanced";
                return false;
            }
            kind[i * NF + f] = (int8_t)kd;
            pos[i * NF + f] = (int8_t)pb;
            if (kd == F_SAME || kd == F_COARSER) {
                nbr[i * NF + f] = sub[0];
            } else if (kd == F_FINER) {
                nbr[i * NF + f] = (int32_t)hang.size();
                for (int j = 0; j < NS; ++j) hang.push_back(sub[j]);
            }
            code |= (uint16_t)(kd << (2 * f));
        }
        cls[i] = code;
    }
    return true;
}

int Mesh::neighbour(int64_t i, int axis, int side, int32_t* out, int* posbits) const {
    const Leaf& lf = leaves[i];
    const int l = lf.level, sh = L - l;
    int64_t cn[3] = {lf.c[0], lf.c[1], lf.c[2]};
    cn[axis] += side;
    const int64_t ncell = (int64_t)base[axis] << l;
    if (cn[axis] < 0 || cn[axis] >= ncell) return F_BOUNDARY;
    // finest cell of the neighbouring level-l cell that touches this face, at its lower tangential corner
    int64_t fc[3];
    for (int k = 0; k < 3; ++k) fc[k] = (k < dim) ? (cn[k] << sh) : 0;
    if (side < 0) fc[axis] = ((cn[axis] + 1) << sh) - 1;
    const int32_t o = leaf_of(fc);
    const int lo = leaves[o].level;
    int tg[2], nt = 0;
    for (int k = 0; k < dim; ++k)
        if (k != axis) tg[nt++] = k;
    if (lo == l) {
        out[0] = o;
        *posbits = 0;
        return F_SAME;
    }
    if (lo == l - 1) {
        out[0] = o;
        int pb = 0;
        for (int t = 0; t < nt; ++t) pb |= (lf.c[tg[t]] & 1) << t;
        *posbits = pb;
        return F_COARSER;
    }
    if (lo != l + 1) return -1;
    // finer: the 2^(dim-1) children of cell cn that touch this face
    const int shc = sh - 1;
    for (int b = 0; b < nsub(); ++b) {
        int64_t ch[3] = {0, 0, 0};
        ch[axis] = 2 * cn[axis] + (side > 0 ? 0 : 1);
        for (int t = 0; t < nt; ++t) ch[tg[t]] = 2 * (int64_t)lf.c[tg[t]] + ((b >> t) & 1);
        int64_t f2[3];
        for (int k = 0; k < 3; ++k) f2[k] = (k < dim) ? (ch[k] << shc) : 0;
        const int32_t oc = leaf_of(f2);
        if (leaves[oc].level != l + 1) return -1;
        out[b] = oc;
    }
    *posbits = 0;
    return F_FINER;
}

}  // namespace mdl
