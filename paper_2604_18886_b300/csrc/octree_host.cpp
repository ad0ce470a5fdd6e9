// Host-side octree construction for libocg (Sec. 3 of the paper: leaf / inner cells,
// face 2:1 level restriction).  Refinement flags live in dense per-depth grids; the
// 2:1 rule is closed bottom-up (an inner cell at depth e needs its six face neighbours
// at depth e, i.e. their parents at depth e-1 must be inner); octet tables follow.
//
// Compiled without floating-point contraction so the refinement predicate evaluates
// exactly the float64 expressions documented in ocg.h.
#include "octree_host.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace ocg {

uint64_t morton3(uint64_t i, uint64_t j, uint64_t k) {
    auto spread = [](uint64_t v) {
        v &= 0x1fffffULL;
        v = (v | (v << 32)) & 0x1f00000000ffffULL;
        v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
        v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
        v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
        v = (v | (v << 2)) & 0x1249249249249249ULL;
        return v;
    };
    return spread(i) | (spread(j) << 1) | (spread(k) << 2);
}

void demorton3(uint64_t key, uint64_t& i, uint64_t& j, uint64_t& k) {
    auto compact = [](uint64_t v) {
        v &= 0x1249249249249249ULL;
        v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
        v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
        v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
        v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
        v = (v ^ (v >> 32)) & 0x1fffffULL;
        return v;
    };
    i = compact(key);
    j = compact(key >> 1);
    k = compact(key >> 2);
}

static inline int64_t lex(int64_t i, int64_t j, int64_t k, int64_t n) { return (k * n + j) * n + i; }

// Refinement predicate (documented in ocg.h); no FMA contraction in this file.
static bool refine_pred(const ocg_octree_desc& d, int depth, int64_t i, int64_t j, int64_t k) {
    const double nd = (double)((int64_t)d.n0 << depth);
    const double x = ((double)i + 0.5) / nd;
    const double y = ((double)j + 0.5) / nd;
    const double z = ((double)k + 0.5) / nd;
    if (d.refine == OCG_REFINE_BALL_CENTRE) {
        const double dx = x - d.spheres[0][0], dy = y - d.spheres[0][1], dz = z - d.spheres[0][2];
        const double r = d.spheres[0][3];
        const double s = dx * dx + dy * dy;
        return (s + dz * dz) < r * r;
    }
    if (d.refine == OCG_REFINE_SDF_BAND) {
        double phi = INFINITY;
        for (int q = 0; q < d.n_spheres; ++q) {
            const double dx = x - d.spheres[q][0], dy = y - d.spheres[q][1], dz = z - d.spheres[q][2];
            const double s = dx * dx + dy * dy;
            const double v = std::sqrt(s + dz * dz) - d.spheres[q][3];
            phi = std::fmin(phi, v);
        }
        for (int q = 0; q < d.n_boxes; ++q) {
            const double* b = d.boxes[q];
            const double qx = std::fabs(x - 0.5 * (b[0] + b[3])) - 0.5 * (b[3] - b[0]);
            const double qy = std::fabs(y - 0.5 * (b[1] + b[4])) - 0.5 * (b[4] - b[1]);
            const double qz = std::fabs(z - 0.5 * (b[2] + b[5])) - 0.5 * (b[5] - b[2]);
            const double mx = std::fmax(qx, 0.0), my = std::fmax(qy, 0.0), mz = std::fmax(qz, 0.0);
            const double s = mx * mx + my * my;
            const double outside = std::sqrt(s + mz * mz);
            const double inside = std::fmin(std::fmax(qx, std::fmax(qy, qz)), 0.0);
            phi = std::fmin(phi, outside + inside);
        }
        const double slack = d.band + (0.5 * std::sqrt(3.0)) * (1.0 / nd);
        return std::fabs(phi) < slack;
    }
    return false;
}

int64_t HostTree::cell_index(int m, int64_t i, int64_t j, int64_t k) const {
    if (m < mc || m > D) return -1;
    const LevelMeta& l = L(m);
    if (i < 0 || j < 0 || k < 0 || i >= l.N || j >= l.N || k >= l.N) return -1;
    const int slot = (int)((i & 1) | ((j & 1) << 1) | ((k & 1) << 2));
    if (l.ni > 0) return l.off + 8 * lex(i >> 1, j >> 1, k >> 1, l.ni) + slot;
    const auto& ok = okeys[m - mc];
    const uint64_t key = morton3(i >> 1, j >> 1, k >> 1);
    auto it = std::lower_bound(ok.begin(), ok.end(), key);
    if (it == ok.end() || *it != key) return -1;
    const int64_t o = it - ok.begin();
    return l.off + 8 * o + ((i & 1) | ((j & 1) << 1) | ((k & 1) << 2));
}

void HostTree::cell_coords(int m, int64_t g, int64_t& i, int64_t& j, int64_t& k) const {
    const LevelMeta& l = L(m);
    const int64_t lc = g - l.off;
    uint64_t I, J, K;
    if (l.ni > 0) {
        const int64_t o = lc >> 3;
        I = o % l.ni;
        J = (o / l.ni) % l.ni;
        K = o / ((int64_t)l.ni * l.ni);
    } else {
        demorton3(okeys[m - mc][lc >> 3], I, J, K);
    }
    const int s = (int)(lc & 7);
    i = 2 * (int64_t)I + (s & 1);
    j = 2 * (int64_t)J + ((s >> 1) & 1);
    k = 2 * (int64_t)K + ((s >> 2) & 1);
}

static int sub_index(int a, int s) {
    // position of slot s among the 4 cells of an octet face normal to axis a
    if (a == 0) return ((s >> 1) & 1) | (((s >> 2) & 1) << 1);
    if (a == 1) return (s & 1) | (((s >> 2) & 1) << 1);
    return (s & 1) | (((s >> 1) & 1) << 1);
}

void build_host_tree(const ocg_octree_desc& desc, HostTree& T) {
    T.desc = desc;
    const int n0 = desc.n0, D = desc.max_depth;
    if (n0 < 2 || (n0 & 1)) throw std::runtime_error("n0 must be even and >= 2");
    if (D < 0 || D > 12) throw std::runtime_error("max_depth out of range [0, 12]");
    if (((int64_t)n0 << D) > (1 << 20)) throw std::runtime_error("n0 * 2^max_depth exceeds 2^20");
    if (desc.refine < OCG_REFINE_NONE || desc.refine > OCG_REFINE_SDF_BAND)
        throw std::runtime_error("unknown refine kind");
    if (desc.n_spheres < 0 || desc.n_spheres > 4 || desc.n_boxes < 0 || desc.n_boxes > 4)
        throw std::runtime_error("too many primitives");
    if (desc.refine == OCG_REFINE_BALL_CENTRE && desc.n_spheres < 1)
        throw std::runtime_error("ball-centre refinement needs one sphere");
    T.n0 = n0;
    T.D = D;
    int N = n0, mc = 0;
    while (N % 2 == 0 && N > 4) { N /= 2; --mc; }
    T.mc = mc;
    const int Nc = N, Ncp = N + (N & 1);
    if ((int64_t)Ncp * Ncp * Ncp > 64 * 64 * 64) throw std::runtime_error("coarsest grid too large");

    // ---- refinement flags per depth (dense, lexicographic)
    std::vector<std::vector<uint8_t>> ref(D + 1);
    for (int d = 0; d < D; ++d) {
        const int64_t nd = (int64_t)n0 << d;
        ref[d].assign(nd * nd * nd, 0);
        auto& R = ref[d];
        const std::vector<uint8_t>* P = d > 0 ? &ref[d - 1] : nullptr;
        const int64_t np = nd / 2;
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nd; ++k)
            for (int64_t j = 0; j < nd; ++j)
                for (int64_t i = 0; i < nd; ++i) {
                    if (P && !(*P)[lex(i >> 1, j >> 1, k >> 1, np)]) continue;
                    if (refine_pred(desc, d, i, j, k)) R[lex(i, j, k, nd)] = 1;
                }
    }
    // ---- face 2:1 balance, deepest inner cells first
    for (int e = D - 1; e >= 1; --e) {
        const int64_t ne = (int64_t)n0 << e, np = ne / 2;
        auto& R = ref[e];
        auto& Rp = ref[e - 1];
        for (int64_t k = 0; k < ne; ++k)
            for (int64_t j = 0; j < ne; ++j)
                for (int64_t i = 0; i < ne; ++i) {
                    if (!R[lex(i, j, k, ne)]) continue;
                    const int64_t c[3] = {i, j, k};
                    for (int a = 0; a < 3; ++a)
                        for (int s = -1; s <= 1; s += 2) {
                            int64_t q[3] = {c[0], c[1], c[2]};
                            q[a] += s;
                            if (q[a] < 0 || q[a] >= ne) continue;
                            Rp[lex(q[0] >> 1, q[1] >> 1, q[2] >> 1, np)] = 1;
                        }
                }
    }
    auto refined = [&](int d, int64_t i, int64_t j, int64_t k) -> bool {
        if (d >= D) return false;
        const int64_t nd = (int64_t)n0 << d;
        return ref[d][lex(i, j, k, nd)] != 0;
    };

    // ---- levels and octet parent keys
    const int nlev = D - mc + 1;
    T.lv.assign(nlev, LevelMeta{});
    T.okeys.assign(nlev, {});
    for (int m = mc; m <= D; ++m) {
        LevelMeta& l = T.L(m);
        l.m = m;
        if (m >= 0) {
            l.N = n0 << m;
            l.Np = l.N;
            l.h = 1.0 / (double)l.N;
        } else {
            l.N = n0 >> (-m);
            l.Np = (m == mc) ? Ncp : l.N;
        }
        auto& keys = T.okeys[m - mc];
        if (m >= 1) {
            const int64_t np = (int64_t)n0 << (m - 1);
            const auto& R = ref[m - 1];
            for (int64_t k = 0; k < np; ++k)
                for (int64_t j = 0; j < np; ++j)
                    for (int64_t i = 0; i < np; ++i)
                        if (R[lex(i, j, k, np)]) keys.push_back(morton3(i, j, k));
            std::sort(keys.begin(), keys.end());
            l.noct = (int64_t)keys.size();
        } else {
            l.ni = l.Np / 2;
            l.noct = (int64_t)l.ni * l.ni * l.ni;
        }
        l.ncell = 8 * l.noct;
    }
    T.order.clear();
    for (int m = 0; m <= D; ++m) T.order.push_back(m);
    for (int m = -1; m >= mc; --m) T.order.push_back(m);
    int64_t off = 0;
    for (int m : T.order) {
        LevelMeta& l = T.L(m);
        l.off = off;
        l.oct_off = off / 8;
        off += l.ncell;
        if (m == D) T.ntree = off;
    }
    T.ncell = off;
    T.noct = off / 8;
    if (T.ncell >= (int64_t)1 << 31) throw std::runtime_error("more than 2^31 cells");

    // ---- per-cell tables
    T.child_oct.assign(T.ncell, -1);
    T.cell_rank.assign(T.ncell, -1);
    T.cell_flags.assign(T.ncell, 0);
    T.cell_level.assign(T.ncell, 0);
    for (int m = mc; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
#pragma omp parallel for schedule(static)
        for (int64_t lc = 0; lc < l.ncell; ++lc) {
            const int64_t g = l.off + lc;
            int64_t i, j, k;
            T.cell_coords(m, g, i, j, k);
            T.cell_level[g] = (int8_t)m;
            const bool real = i < l.N && j < l.N && k < l.N;
            if (!real) continue;
            uint8_t fl = 2;
            bool has_children;
            if (m >= 0) {
                has_children = refined(m, i, j, k);
                if (!has_children) fl |= 1;
            } else {
                has_children = true;
            }
            T.cell_flags[g] = fl;
            if (has_children) {
                const LevelMeta& lf = T.L(m + 1);
                if (lf.ni > 0) {
                    T.child_oct[g] = (int32_t)(lf.oct_off + lex(i, j, k, lf.ni));
                } else {
                    const auto& ck = T.okeys[m + 1 - mc];
                    auto it = std::lower_bound(ck.begin(), ck.end(), morton3(i, j, k));
                    T.child_oct[g] = (int32_t)(lf.oct_off + (it - ck.begin()));
                }
            }
        }
    }
    // canonical leaves: sorted by (depth, Morton key)
    T.leaf_cell.clear();
    T.leaf_depth.clear(); T.leaf_i.clear(); T.leaf_j.clear(); T.leaf_k.clear();
    for (int m = 0; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
        std::vector<std::pair<uint64_t, int64_t>> lv;
        for (int64_t lc = 0; lc < l.ncell; ++lc) {
            const int64_t g = l.off + lc;
            if (!(T.cell_flags[g] & 1)) continue;
            int64_t i, j, k;
            T.cell_coords(m, g, i, j, k);
            lv.push_back({morton3(i, j, k), g});
        }
        std::sort(lv.begin(), lv.end());
        for (const auto& e : lv) {
            const int64_t g = e.second;
            int64_t i, j, k;
            T.cell_coords(m, g, i, j, k);
            T.cell_rank[g] = (int32_t)T.leaf_cell.size();
            T.leaf_cell.push_back((int32_t)g);
            T.leaf_depth.push_back(m);
            T.leaf_i.push_back((int32_t)i); T.leaf_j.push_back((int32_t)j); T.leaf_k.push_back((int32_t)k);
        }
    }
    T.nleaf = (int64_t)T.leaf_cell.size();

    // ---- octet tables: neighbours, parents, T records
    T.nbr.assign(6 * T.noct, -1);
    T.oct_parent.assign(T.noct, -1);
    T.t_oct.clear();
    T.trec.assign(T.noct, -1);
    auto& trec = T.trec;
    for (int m = mc; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
        const int64_t PG = m >= 1 ? ((int64_t)n0 << (m - 1)) : l.Np / 2;
        const auto& keys = T.okeys[m - mc];
        for (int64_t o = 0; o < l.noct; ++o) {
            uint64_t I, J, K;
            if (l.ni > 0) {
                I = o % l.ni;
                J = (o / l.ni) % l.ni;
                K = o / ((int64_t)l.ni * l.ni);
            } else {
                demorton3(keys[o], I, J, K);
            }
            const int64_t go = l.oct_off + o;
            if (m > mc) T.oct_parent[go] = (int32_t)T.cell_index(m - 1, I, J, K);
            const int64_t P[3] = {(int64_t)I, (int64_t)J, (int64_t)K};
            for (int a = 0; a < 3; ++a)
                for (int sd = 0; sd < 2; ++sd) {
                    const int dir = 2 * a + sd;
                    int64_t q[3] = {P[0], P[1], P[2]};
                    q[a] += sd ? 1 : -1;
                    int32_t v = -1;
                    if (q[a] >= 0 && q[a] < PG) {
                        const bool inner = (m <= 0) || refined(m - 1, q[0], q[1], q[2]);
                        if (l.ni > 0) {
                            v = (int32_t)lex(q[0], q[1], q[2], l.ni);
                        } else if (inner) {
                            auto it = std::lower_bound(keys.begin(), keys.end(), morton3(q[0], q[1], q[2]));
                            v = (int32_t)(it - keys.begin());
                        } else {
                            const int64_t Kc = T.cell_index(m - 1, q[0], q[1], q[2]);
                            if (Kc < 0 || !(T.cell_flags[Kc] & 1))
                                throw std::runtime_error("internal: unbalanced T-junction");
                            if (trec[go] < 0) {
                                trec[go] = (int32_t)T.t_oct.size();
                                T.t_oct.push_back((int32_t)go);
                            }
                            v = (int32_t)(-2 - Kc);
                        }
                    }
                    T.nbr[(int64_t)dir * T.noct + go] = v;
                }
        }
    }
    T.nt = (int64_t)T.t_oct.size();

    // ---- neighbour export and canonical faces
    T.nb_kind.assign(6 * T.nleaf, 0);
    T.nb_rank.assign(6 * T.nleaf, -1);
    struct F { int32_t a, d, i, j, k; int64_t minus, plus, slot; uint8_t kind; uint64_t mk; };
    std::vector<F> faces;
    for (int64_t r = 0; r < T.nleaf; ++r) {
        const int d = T.leaf_depth[r];
        const int64_t c[3] = {T.leaf_i[r], T.leaf_j[r], T.leaf_k[r]};
        const int64_t nd = (int64_t)n0 << d;
        const int64_t g = T.leaf_cell[r];
        const int s = (int)((g - T.L(d).off) & 7);
        for (int a = 0; a < 3; ++a)
            for (int sd = 0; sd < 2; ++sd) {
                const int dir = 2 * a + sd;
                int64_t q[3] = {c[0], c[1], c[2]};
                q[a] += sd ? 1 : -1;
                int8_t kind = 0;
                int64_t rk = -1;
                if (q[a] >= 0 && q[a] < nd) {
                    const int64_t gn = T.cell_index(d, q[0], q[1], q[2]);
                    if (gn >= 0) {
                        if (T.cell_flags[gn] & 1) { kind = 1; rk = T.cell_rank[gn]; }
                        else kind = 3;
                    } else {
                        const int64_t gk = T.cell_index(d - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1);
                        kind = 2;
                        rk = T.cell_rank[gk];
                    }
                }
                T.nb_kind[6 * r + dir] = kind;
                T.nb_rank[6 * r + dir] = rk;
                if (sd == 0 && (kind == 1 || kind == 2)) {
                    faces.push_back({a, d, (int32_t)c[0], (int32_t)c[1], (int32_t)c[2], rk, r,
                                     (int64_t)a * T.ncell + g, 0, morton3(c[0], c[1], c[2])});
                }
                if (sd == 1 && kind == 2) {
                    const int64_t go = (g >> 3);
                    const int32_t t = T.trec[go];
                    const int64_t slot = (int64_t)(dir * 4 + sub_index(a, s)) * T.nt + t;
                    faces.push_back({a, d, (int32_t)q[0], (int32_t)q[1], (int32_t)q[2], r, rk, slot, 1,
                                     morton3(q[0], q[1], q[2])});
                }
            }
    }
    std::sort(faces.begin(), faces.end(), [](const F& x, const F& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.d != y.d) return x.d < y.d;
        return x.mk < y.mk;
    });
    T.nface = (int64_t)faces.size();
    T.f_axis.resize(T.nface); T.f_depth.resize(T.nface);
    T.f_i.resize(T.nface); T.f_j.resize(T.nface); T.f_k.resize(T.nface);
    T.f_minus.resize(T.nface); T.f_plus.resize(T.nface);
    T.f_slot.resize(T.nface); T.f_kind.resize(T.nface);
    for (int64_t f = 0; f < T.nface; ++f) {
        const F& x = faces[f];
        T.f_axis[f] = x.a; T.f_depth[f] = x.d; T.f_i[f] = x.i; T.f_j[f] = x.j; T.f_k[f] = x.k;
        T.f_minus[f] = x.minus; T.f_plus[f] = x.plus; T.f_slot[f] = x.slot; T.f_kind[f] = x.kind;
    }
}

// ---------------------------------------------------------------- adjoint tables
namespace {

// Leaves under cell g with their averaging weights (1/8 per level below g).
void collect_support(const HostTree& T, int64_t g, double w, std::vector<std::pair<int32_t, double>>& out) {
    const int32_t co = T.child_oct[g];
    if (co < 0) {
        out.push_back({(int32_t)g, w});
        return;
    }
    for (int s = 0; s < 8; ++s) collect_support(T, 8 * (int64_t)co + s, w * 0.125, out);
}

bool fine_is_minus(const HostTree& T, int64_t f) {
    return T.leaf_depth[T.f_minus[f]] == T.f_depth[f];
}

}  // namespace

void build_transpose_correction(const HostTree& T, TransposeCorrection& out) {
    struct E {
        int32_t row, col, face;
        double mult;
    };
    std::vector<E> e;
    std::vector<std::pair<int32_t, double>> supp;
    for (int64_t f = 0; f < T.nface; ++f) {
        const int64_t rm = T.f_minus[f], rp = T.f_plus[f];
        if (T.leaf_depth[rm] == T.leaf_depth[rp]) continue;
        const bool fm = fine_is_minus(T, f);
        const int32_t gi = T.leaf_cell[fm ? rm : rp];
        const int32_t gK = T.leaf_cell[fm ? rp : rm];
        const int64_t gP = T.oct_parent[gi >> 3];
        const double hh = 0.5 / (double)((int64_t)T.n0 << T.f_depth[f]);
        supp.clear();
        collect_support(T, gP, 1.0, supp);
        const int32_t fi = (int32_t)f;
        e.push_back({gi, gK, fi, hh});
        e.push_back({gK, gi, fi, -hh});
        for (const auto& jw : supp) {
            const double a = hh * jw.second;
            e.push_back({gi, jw.first, fi, -a});
            e.push_back({gK, jw.first, fi, a});
            e.push_back({jw.first, gi, fi, a});
            e.push_back({jw.first, gK, fi, -a});
        }
    }
    std::stable_sort(e.begin(), e.end(), [](const E& x, const E& y) { return x.row < y.row; });
    out = TransposeCorrection{};
    out.col.resize(e.size());
    out.face.resize(e.size());
    out.mult.resize(e.size());
    for (size_t q = 0; q < e.size(); ++q) {
        if (q == 0 || e[q].row != e[q - 1].row) {
            out.row.push_back(e[q].row);
            out.ptr.push_back((int32_t)q);
        }
        out.col[q] = e[q].col;
        out.face[q] = e[q].face;
        out.mult[q] = e[q].mult;
    }
    out.ptr.push_back((int32_t)e.size());
}

void build_face_grad_tables(const HostTree& T, std::vector<int32_t>& fa, std::vector<int32_t>& fb,
                            std::vector<int32_t>& fp, std::vector<double>& fh) {
    fa.resize(T.nface);
    fb.resize(T.nface);
    fp.resize(T.nface);
    fh.resize(T.nface);
    for (int64_t f = 0; f < T.nface; ++f) {
        const int64_t rm = T.f_minus[f], rp = T.f_plus[f];
        fh[f] = 1.0 / (double)((int64_t)T.n0 << T.f_depth[f]);
        if (T.leaf_depth[rm] == T.leaf_depth[rp]) {
            fa[f] = T.leaf_cell[rm];
            fb[f] = T.leaf_cell[rp];
            fp[f] = -1;
        } else {
            const bool fm = fine_is_minus(T, f);
            fa[f] = T.leaf_cell[fm ? rm : rp];
            fb[f] = T.leaf_cell[fm ? rp : rm];
            fp[f] = T.oct_parent[fa[f] >> 3];
        }
    }
}

}  // namespace ocg
