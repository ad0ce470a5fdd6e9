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
#include <utility>

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

// Deterministic sine and cosine of the sine-band predicate (the exact recipe is stated in
// ocg.h): Cody-Waite reduction by pi/2 with a three-part constant whose first two parts
// carry 33 significant bits (k * part is exact for |k| < 2^20), then Taylor polynomials of
// the reduced argument r in [-pi/4, pi/4] evaluated by Horner's rule; the truncation error
// there is below 1e-19.  Coefficients are (-1)^j / n!, formed by one IEEE division of the
// exactly representable factorial.
namespace {
struct DetTrig {
    double sc[8];   // r^(2j+3) coefficient of sin r, j = 0..7
    double cc[9];   // r^(2j+2) coefficient of cos r, j = 0..8
    DetTrig() {
        double f = 1.0;
        for (int n = 1; n <= 18; ++n) {
            f = f * (double)n;   // exact: 18! < 2^53
            if (n >= 3 && (n & 1)) sc[(n - 3) / 2] = (((n - 3) / 2) & 1 ? 1.0 : -1.0) / f;
            if (n >= 2 && !(n & 1)) cc[(n - 2) / 2] = (((n - 2) / 2) & 1 ? 1.0 : -1.0) / f;
        }
    }
};
const DetTrig& det_trig() {
    static const DetTrig t;
    return t;
}
constexpr double DT_2_OVER_PI = 0x1.45f306dc9c883p-1;
constexpr double DT_P1 = 0x1.921fb544p+0;
constexpr double DT_P2 = 0x1.0b4611a6p-34;
constexpr double DT_P3 = 0x1.3198a2e037073p-69;
constexpr double DT_TWO_PI = 0x1.921fb54442d18p+2;

// sin and cos of a together (the predicate needs both at the same argument)
void det_sincos(double a, double& sa, double& ca) {
    const DetTrig& T = det_trig();
    const double k = std::rint(a * DT_2_OVER_PI);
    const double r = ((a - k * DT_P1) - k * DT_P2) - k * DT_P3;
    const double r2 = r * r;
    double ps = T.sc[7];
    for (int j = 6; j >= 0; --j) ps = ps * r2 + T.sc[j];
    double pc = T.cc[8];
    for (int j = 7; j >= 0; --j) pc = pc * r2 + T.cc[j];
    const double s = r + (r * r2) * ps;
    const double c = 1.0 + r2 * pc;
    switch ((int)((int64_t)k & 3)) {
        case 0: sa = s; ca = c; break;
        case 1: sa = c; ca = -s; break;
        case 2: sa = -s; ca = -c; break;
        default: sa = -c; ca = s; break;
    }
}
}  // namespace

// Signed distance of the fluid region for OCG_REFINE_SDF_BAND (positive in fluid, negative
// in the solids): min over the spheres |x - c| - r and the boxes' signed distances.
double solid_sdf(const ocg_octree_desc& d, double x, double y, double z) {
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
    return phi;
}

// Area fraction of {phi > 0} on a triangle where phi is linear with vertex values a, b, c.
static double tri_positive_fraction(double a, double b, double c) {
    double lo = a, mid = b, hi = c;
    if (lo > mid) std::swap(lo, mid);
    if (mid > hi) std::swap(mid, hi);
    if (lo > mid) std::swap(lo, mid);
    if (lo > 0.0) return 1.0;
    if (hi > 0.0 && mid <= 0.0) return hi * hi / ((hi - lo) * (hi - mid));       // one corner positive
    if (mid > 0.0 && lo <= 0.0) return 1.0 - lo * lo / ((mid - lo) * (hi - lo)); // one corner negative
    return 0.0;
}

float face_beta_geometric(const ocg_octree_desc& d, int m, int axis, int64_t i, int64_t j, int64_t k) {
    const double h = 1.0 / ((double)d.n0 * std::ldexp(1.0, m));
    const double base[3] = {(double)i * h, (double)j * h, (double)k * h};
    const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;
    auto corner = [&](int du, int dv) {
        double q[3] = {base[0], base[1], base[2]};
        q[u] = q[u] + (du ? h : 0.0);
        q[v] = q[v] + (dv ? h : 0.0);
        return solid_sdf(d, q[0], q[1], q[2]);
    };
    const double p00 = corner(0, 0), p10 = corner(1, 0), p11 = corner(1, 1), p01 = corner(0, 1);
    const double t1 = tri_positive_fraction(p00, p10, p11);
    const double t2 = tri_positive_fraction(p00, p11, p01);
    const double f = 0.5 * (t1 + t2);
    return (float)std::fmin(std::fmax(f, 1e-3), 1.0);
}

// The star function of Sec. 4.1 (documented in ocg.h): r - (r0 + (a T_k(dz/r)) T_k(dx/rho))
// about spheres[0]'s centre, T_k by the Chebyshev recurrence.
static double star_phi(const ocg_octree_desc& d, double x, double y, double z) {
    const double dx = x - d.spheres[0][0], dy = y - d.spheres[0][1], dz = z - d.spheres[0][2];
    const double rho2 = dx * dx + dy * dy;
    const double r = std::sqrt(rho2 + dz * dz), rho = std::sqrt(rho2);
    const double u = r > 0.0 ? dz / r : 1.0, v = rho > 0.0 ? dx / rho : 1.0;
    const int k = (int)d.spheres[1][1];
    auto cheb = [k](double w) {
        double t0 = 1.0, t1 = w;
        if (k == 0) return t0;
        for (int n = 2; n <= k; ++n) {
            const double t = (2.0 * w) * t1 - t0;
            t0 = t1;
            t1 = t;
        }
        return t1;
    };
    return r - (d.spheres[0][3] + (d.spheres[1][0] * cheb(u)) * cheb(v));
}

// Refinement predicate (documented in ocg.h); no FMA contraction in this file.
static bool refine_pred(const ocg_octree_desc& d, int depth, int64_t i, int64_t j, int64_t k) {
    // tiles of 2^t cells per axis decide together, as the depth-(depth - t) cell that covers
    // them: its centre and size (nd cells per axis; exact, n0 is a multiple of 2^t)
    const int t = d.tile_log2;
    i >>= t;
    j >>= t;
    k >>= t;
    const double nd = (double)(((int64_t)d.n0 << depth) >> t);
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
        if (t > 0) {
            // a tile meets the band of a sphere when the sphere's signed distance takes a
            // value in (-band, band) on the closed box: its range there is
            // [dmin - r, dmax - r], dmin / dmax the nearest / farthest distance from the
            // centre to the box; boxes keep the centre test with the tile's half-diagonal
            const double lo[3] = {(double)i / nd, (double)j / nd, (double)k / nd};
            const double hi[3] = {((double)i + 1.0) / nd, ((double)j + 1.0) / nd, ((double)k + 1.0) / nd};
            for (int q = 0; q < d.n_spheres; ++q) {
                double n2 = 0.0, f2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double c = d.spheres[q][a];
                    const double nc = c < lo[a] ? lo[a] : (c > hi[a] ? hi[a] : c);
                    const double dn = nc - c;
                    const double df = std::fmax(std::fabs(lo[a] - c), std::fabs(hi[a] - c));
                    n2 = n2 + dn * dn;
                    f2 = f2 + df * df;
                }
                const double r = d.spheres[q][3];
                if (std::sqrt(n2) - r < d.band && std::sqrt(f2) - r > -d.band) return true;
            }
            if (d.n_boxes == 0) return false;
            ocg_octree_desc bx = d;
            bx.n_spheres = 0;
            const double phi = solid_sdf(bx, x, y, z);
            return std::fabs(phi) < d.band + (0.5 * std::sqrt(3.0)) * (1.0 / nd);
        }
        const double phi = solid_sdf(d, x, y, z);
        const double slack = d.band + (0.5 * std::sqrt(3.0)) * (1.0 / nd);
        return std::fabs(phi) < slack;
    }
    if (d.refine == OCG_REFINE_STAR_BAND) {
        if (t > 0) {
            // a tile meets the band when the star function takes a value below band and one
            // above -band among its 27 lattice points (corners, edge and face midpoints,
            // centre): (i + q/2) / nd, q = 0, 1, 2 per axis
            double lo = INFINITY, hi = -INFINITY;
            for (int qz = 0; qz < 3; ++qz)
                for (int qy = 0; qy < 3; ++qy)
                    for (int qx = 0; qx < 3; ++qx) {
                        const double px = ((double)i + 0.5 * qx) / nd, py = ((double)j + 0.5 * qy) / nd,
                                     pz = ((double)k + 0.5 * qz) / nd;
                        const double f = star_phi(d, px, py, pz);
                        lo = std::fmin(lo, f);
                        hi = std::fmax(hi, f);
                    }
            return lo < d.band && hi > -d.band;
        }
        const double phi = star_phi(d, x, y, z);
        const double slack = d.band + (d.spheres[1][2] * (0.5 * std::sqrt(3.0))) * (1.0 / nd);
        return std::fabs(phi) < slack;
    }
    if (d.refine == OCG_REFINE_SINE_BAND) {
        double s = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int w = 0; w < d.n_sines; ++w) {
            const double* q = d.sines[w];
            const double w2 = DT_TWO_PI * q[0];
            const double a = w2 * ((q[1] * x + q[2] * y) + q[3] * z) + q[4];
            double sa, ca;
            det_sincos(a, sa, ca);
            s = s + sa;
            const double g = w2 * ca;
            gx = gx + g * q[1];
            gy = gy + g * q[2];
            gz = gz + g * q[3];
        }
        const double n = (double)d.n_sines;
        const double phi = s / n;
        const double gn = std::sqrt((gx * gx + gy * gy) + gz * gz) / n;
        const double slack = d.band + (gn * (0.5 * std::sqrt(3.0))) * (1.0 / nd);
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

// Parallel stream compaction: out = [value(c) for c in 0..n-1 if keep(c)], in order.
// pred(c, value&) returns keep and fills value.
template <class V, class F>
static std::vector<V> par_compact(int64_t n, F&& pred) {
#ifdef _OPENMP
    const int nch = std::max(1, omp_get_max_threads() * 8);
#else
    const int nch = 1;
#endif
    std::vector<int64_t> cnt(nch + 1, 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nch; ++c) {
        const int64_t lo = n * c / nch, hi = n * (c + 1) / nch;
        int64_t k = 0;
        V v{};
        for (int64_t q = lo; q < hi; ++q) k += pred(q, v) ? 1 : 0;
        cnt[c + 1] = k;
    }
    for (int c = 0; c < nch; ++c) cnt[c + 1] += cnt[c];
    std::vector<V> out(cnt[nch]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nch; ++c) {
        const int64_t lo = n * c / nch, hi = n * (c + 1) / nch;
        int64_t k = cnt[c];
        V v{};
        for (int64_t q = lo; q < hi; ++q)
            if (pred(q, v)) out[k++] = v;
    }
    return out;
}

// Parallel exclusive scan: visit(c, sum of weight(0..c-1)) for every c, in chunks.
template <class W, class F>
static void par_scan(int64_t n, W&& weight, F&& visit) {
#ifdef _OPENMP
    const int nch = std::max(1, omp_get_max_threads() * 8);
#else
    const int nch = 1;
#endif
    std::vector<int64_t> cnt(nch + 1, 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nch; ++c) {
        const int64_t lo = n * c / nch, hi = n * (c + 1) / nch;
        int64_t k = 0;
        for (int64_t q = lo; q < hi; ++q) k += weight(q);
        cnt[c + 1] = k;
    }
    for (int c = 0; c < nch; ++c) cnt[c + 1] += cnt[c];
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nch; ++c) {
        const int64_t lo = n * c / nch, hi = n * (c + 1) / nch;
        int64_t k = cnt[c];
        for (int64_t q = lo; q < hi; ++q) {
            visit(q, k);
            k += weight(q);
        }
    }
}

static int sub_index(int a, int s) {
    // position of slot s among the 4 cells of an octet face normal to axis a
    if (a == 0) return ((s >> 1) & 1) | (((s >> 2) & 1) << 1);
    if (a == 1) return (s & 1) | (((s >> 2) & 1) << 1);
    return (s & 1) | (((s >> 1) & 1) << 1);
}

static void build_impl(const ocg_octree_desc& desc, HostTree& T, const HostTree* prev, const double* box);

void build_host_tree(const ocg_octree_desc& desc, HostTree& T) { build_impl(desc, T, nullptr, nullptr); }

void rebuild_host_tree(const HostTree& prev, const ocg_octree_desc& desc, const double box[6], HostTree& T) {
    if (desc.n0 != prev.desc.n0 || desc.max_depth != prev.desc.max_depth || desc.refine != prev.desc.refine ||
        desc.tile_log2 != prev.desc.tile_log2)
        throw std::runtime_error("rebuild: n0, max_depth, refine and tile_log2 must equal the previous octree's");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(box[a]) || !std::isfinite(box[a + 3]) || box[a] > box[a + 3])
            throw std::runtime_error("rebuild: the box must be finite with lo <= hi on each axis");
    if ((int)prev.pred.size() != std::max(prev.D, 0)) throw std::runtime_error("rebuild: previous octree incomplete");
    build_impl(desc, T, &prev, box);
}

static void build_impl(const ocg_octree_desc& desc, HostTree& T, const HostTree* prev, const double* box) {
    T.desc = desc;
    const int n0 = desc.n0, D = desc.max_depth;
    if (n0 < 2 || (n0 & 1)) throw std::runtime_error("n0 must be even and >= 2");
    if (D < 0 || D > 12) throw std::runtime_error("max_depth out of range [0, 12]");
    if (((int64_t)n0 << D) > (1 << 20)) throw std::runtime_error("n0 * 2^max_depth exceeds 2^20");
    if (desc.refine < OCG_REFINE_NONE || desc.refine > OCG_REFINE_STAR_BAND)
        throw std::runtime_error("unknown refine kind");
    if (desc.refine == OCG_REFINE_STAR_BAND) {
        const double k = desc.spheres[1][1];
        if (desc.n_spheres < 2 || !(k >= 0.0 && k <= 16.0 && k == std::floor(k)) || !(desc.spheres[1][2] >= 0.0))
            throw std::runtime_error("star refinement needs spheres[0] = (c, r0), spheres[1] = (a, k in 0..16, L >= 0)");
    }
    if (desc.refine == OCG_REFINE_SINE_BAND) {
        if (desc.n_sines < 1 || desc.n_sines > 8) throw std::runtime_error("n_sines must be in 1..8");
        for (int w = 0; w < desc.n_sines; ++w) {
            const double* q = desc.sines[w];
            // |a| <= 2 pi |kappa| (|dx| + |dy| + |dz|) + |theta| on the unit cube
            const double amax = 6.3 * std::fabs(q[0]) * (std::fabs(q[1]) + std::fabs(q[2]) + std::fabs(q[3])) +
                                std::fabs(q[4]);
            if (!(amax < 1048576.0)) throw std::runtime_error("sine wave argument out of range (|a| < 2^20)");
        }
    }
    if (desc.tile_log2 < 0 || desc.tile_log2 > 4 || desc.n0 % (1 << desc.tile_log2) != 0)
        throw std::runtime_error("tile_log2 must be in 0..4 with n0 a multiple of 2^tile_log2");
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

    // ---- refinement flags per depth (dense, lexicographic): a cell of depth d is refined
    // when its parent is and the predicate holds.  A rebuild takes a cell's flag from the
    // previous octree when the cell lies outside the changed box and its parent's flag is
    // unchanged (the predicate there is the same by the caller's contract), and evaluates
    // the predicate for every other cell; the index window has one cell of margin.
    std::vector<std::vector<uint8_t>> ref(D + 1);
    for (int d = 0; d < D; ++d) {
        const int64_t nd = (int64_t)n0 << d;
        ref[d].assign(nd * nd * nd, 0);
        auto& R = ref[d];
        const std::vector<uint8_t>* P = d > 0 ? &ref[d - 1] : nullptr;
        const std::vector<uint8_t>* Rold = prev ? &prev->pred[d] : nullptr;
        const std::vector<uint8_t>* Pold = prev && d > 0 ? &prev->pred[d - 1] : nullptr;
        int64_t lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
        if (prev)
            for (int a = 0; a < 3; ++a) {
                lo[a] = (int64_t)std::floor(std::max(-1.0, std::min(2.0, box[a])) * (double)nd) - 1;
                hi[a] = (int64_t)std::floor(std::max(-1.0, std::min(2.0, box[a + 3])) * (double)nd) + 1;
                // whole tiles: a cell's flag is its tile's
                const int tl = desc.tile_log2;
                lo[a] = (lo[a] >> tl) << tl;
                hi[a] = (((hi[a] >> tl) + 1) << tl) - 1;
            }
        const int64_t np = nd / 2;
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nd; ++k)
            for (int64_t j = 0; j < nd; ++j)
                for (int64_t i = 0; i < nd; ++i) {
                    const int64_t pc = lex(i >> 1, j >> 1, k >> 1, np);
                    if (P && !(*P)[pc]) continue;
                    const int64_t c = lex(i, j, k, nd);
                    if (Rold) {
                        const bool inside = i >= lo[0] && i <= hi[0] && j >= lo[1] && j <= hi[1] &&
                                            k >= lo[2] && k <= hi[2];
                        if (!inside && (!Pold || (*Pold)[pc])) {
                            R[c] = (*Rold)[c];
                            continue;
                        }
                    }
                    if (refine_pred(desc, d, i, j, k)) R[c] = 1;
                }
    }
    T.pred.assign(ref.begin(), ref.begin() + std::max(D, 0));
    // ---- face 2:1 balance, deepest inner cells first (within one depth the order of the
    // marks does not matter: depth e is read, depth e-1 written).  With tiles the marks go
    // to whole tiles of depth e-1 (a tile is refined as a unit), collected in TM first.
    const int tl = desc.tile_log2;
    for (int e = D - 1; e >= 1; --e) {
        const int64_t ne = (int64_t)n0 << e, np = ne / 2, nt = np >> tl;
        const auto& R = ref[e];
        std::vector<uint8_t> TM(tl > 0 ? nt * nt * nt : 0, 0);
        uint8_t* Rp = tl > 0 ? TM.data() : ref[e - 1].data();
        const int sh = 1 + tl;   // depth-e coordinate -> parent's tile coordinate
        const int64_t nm = tl > 0 ? nt : np;
#pragma omp parallel for schedule(static)
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
                            __atomic_store_n(&Rp[lex(q[0] >> sh, q[1] >> sh, q[2] >> sh, nm)], (uint8_t)1,
                                             __ATOMIC_RELAXED);
                        }
                }
        if (tl > 0) {
            uint8_t* P = ref[e - 1].data();
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < np; ++k)
                for (int64_t j = 0; j < np; ++j)
                    for (int64_t i = 0; i < np; ++i)
                        if (TM[lex(i >> tl, j >> tl, k >> tl, nt)]) P[lex(i, j, k, np)] = 1;
        }
    }
    auto refined = [&](int d, int64_t i, int64_t j, int64_t k) -> bool {
        if (d >= D) return false;
        const int64_t nd = (int64_t)n0 << d;
        return ref[d][lex(i, j, k, nd)] != 0;
    };

    // ---- levels and octet parent keys.  Level 1's octets are the refined root cells in
    // Morton order; for m >= 2 the cells of level m-1 in storage order are already in
    // Morton order (parent key << 3 | slot), so level m's keys are its refined cells.
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
        if (m == 1) {
            const int64_t np = n0;
            const auto& R = ref[0];
            for (int64_t k = 0; k < np; ++k)
                for (int64_t j = 0; j < np; ++j)
                    for (int64_t i = 0; i < np; ++i)
                        if (R[lex(i, j, k, np)]) keys.push_back(morton3(i, j, k));
            std::sort(keys.begin(), keys.end());
        } else if (m >= 2) {
            const auto& pk = T.okeys[m - 1 - mc];
            const auto& R = ref[m - 1];
            const int64_t nd = (int64_t)n0 << (m - 1);
            auto is_ref = [&](uint64_t key) {
                uint64_t i, j, k;
                demorton3(key, i, j, k);
                return R[lex((int64_t)i, (int64_t)j, (int64_t)k, nd)] != 0;
            };
            keys = par_compact<uint64_t>((int64_t)pk.size() * 8, [&](int64_t c, uint64_t& out) {
                const uint64_t key = (pk[c >> 3] << 3) | (uint64_t)(c & 7);
                out = key;
                return is_ref(key);
            });
        }
        if (m >= 1) {
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
#pragma omp parallel sections
    {
#pragma omp section
        T.child_oct.assign(T.ncell, -1);
#pragma omp section
        T.cell_rank.assign(T.ncell, -1);
#pragma omp section
        T.cell_flags.assign(T.ncell, 0);
#pragma omp section
        T.cell_level.assign(T.ncell, 0);
    }
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
            const bool has_children = m >= 0 ? refined(m, i, j, k) : true;
            if (m >= 0 && !has_children) fl |= 1;
            T.cell_flags[g] = fl;
            if (has_children && m <= 0) {
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
        if (m >= 1 && m < D) {
            // children octets of level m+1 follow the refined cells of level m in storage order
            const int64_t base = T.L(m + 1).oct_off;
            par_scan(l.ncell, [&](int64_t lc) { return (T.cell_flags[l.off + lc] & 1) ? 0 : 1; },
                     [&](int64_t lc, int64_t rank) {
                         if (!(T.cell_flags[l.off + lc] & 1)) T.child_oct[l.off + lc] = (int32_t)(base + rank);
                     });
        }
    }
    // canonical leaves: sorted by (depth, Morton key); level 0 by enumerating the Morton
    // keys of the smallest power-of-two cube that holds the root grid in order (a parallel
    // compaction, no sort), levels m >= 1 are stored in Morton order already
    T.leaf_first.assign(D + 2, 0);
    int64_t side = 1;
    while (side < n0) side <<= 1;
    std::vector<std::pair<uint64_t, int32_t>> lv0 =
        par_compact<std::pair<uint64_t, int32_t>>(side * side * side, [&](int64_t key, std::pair<uint64_t, int32_t>& out) {
            uint64_t i, j, k;
            demorton3((uint64_t)key, i, j, k);
            if (i >= (uint64_t)n0 || j >= (uint64_t)n0 || k >= (uint64_t)n0) return false;
            const int64_t g = T.cell_index(0, (int64_t)i, (int64_t)j, (int64_t)k);
            if (!(T.cell_flags[g] & 1)) return false;
            out = {(uint64_t)key, (int32_t)g};
            return true;
        });
    // leaves per level m >= 1 (stored in Morton order already), then each level's leaves
    // written at their canonical ranks by a parallel scan
    T.leaf_first[1] = (int64_t)lv0.size();
    for (int m = 1; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
        int64_t nl = 0;
#pragma omp parallel for schedule(static) reduction(+ : nl)
        for (int64_t lc = 0; lc < l.ncell; ++lc) nl += T.cell_flags[l.off + lc] & 1;
        T.leaf_first[m + 1] = T.leaf_first[m] + nl;
    }
    T.leaf_cell.resize(T.leaf_first[D + 1]);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < (int64_t)lv0.size(); ++q) T.leaf_cell[q] = lv0[q].second;
    for (int m = 1; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
        const int64_t base = T.leaf_first[m];
        par_scan(l.ncell, [&](int64_t lc) { return (int64_t)(T.cell_flags[l.off + lc] & 1); },
                 [&](int64_t lc, int64_t rank) {
                     if (T.cell_flags[l.off + lc] & 1) T.leaf_cell[base + rank] = (int32_t)(l.off + lc);
                 });
    }
    T.nleaf = (int64_t)T.leaf_cell.size();
    T.leaf_first[D + 1] = T.nleaf;
#pragma omp parallel sections
    {
#pragma omp section
        T.leaf_depth.resize(T.nleaf);
#pragma omp section
        T.leaf_i.resize(T.nleaf);
#pragma omp section
        T.leaf_j.resize(T.nleaf);
#pragma omp section
        T.leaf_k.resize(T.nleaf);
    }
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < T.nleaf; ++r) {
        const int64_t g = T.leaf_cell[r];
        const int m = T.cell_level[g];
        int64_t i, j, k;
        T.cell_coords(m, g, i, j, k);
        T.cell_rank[g] = (int32_t)r;
        T.leaf_depth[r] = m;
        T.leaf_i[r] = (int32_t)i; T.leaf_j[r] = (int32_t)j; T.leaf_k[r] = (int32_t)k;
    }

    // ---- octet tables: parents, neighbours (coarse to fine: an adaptive level reads the
    // neighbours of its parents' level), T records
    T.nbr.assign(6 * T.noct, -1);
    T.oct_parent.assign(T.noct, -1);
    for (int m = mc; m <= D; ++m) {
        const LevelMeta& l = T.L(m);
        if (m <= 0) {
#pragma omp parallel for schedule(static)
            for (int64_t o = 0; o < l.noct; ++o) {
                const int64_t I = o % l.ni, J = (o / l.ni) % l.ni, K = o / ((int64_t)l.ni * l.ni);
                const int64_t go = l.oct_off + o;
                if (m > mc) T.oct_parent[go] = (int32_t)T.cell_index(m - 1, I, J, K);
                const int64_t P[3] = {I, J, K};
                for (int dir = 0; dir < 6; ++dir) {
                    const int a = dir >> 1;
                    int64_t q[3] = {P[0], P[1], P[2]};
                    q[a] += (dir & 1) ? 1 : -1;
                    const bool in = q[a] >= 0 && q[a] < l.ni;
                    T.nbr[(int64_t)dir * T.noct + go] = in ? (int32_t)lex(q[0], q[1], q[2], l.ni) : -1;
                }
            }
            continue;
        }
        const LevelMeta& lp = T.L(m - 1);
#pragma omp parallel for schedule(static)
        for (int64_t lc = 0; lc < lp.ncell; ++lc) {
            const int32_t co = T.child_oct[lp.off + lc];
            if (co >= 0) T.oct_parent[co] = (int32_t)(lp.off + lc);
        }
        int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int64_t o = 0; o < l.noct; ++o) {
            const int64_t go = l.oct_off + o;
            const int64_t Pc = T.oct_parent[go];
            const int sp = (int)(Pc & 7);
            const int64_t pog = Pc >> 3;
            for (int dir = 0; dir < 6; ++dir) {
                const int a = dir >> 1, bit = 1 << a;
                const bool plus = dir & 1;
                int64_t Q = -1;
                if (((sp & bit) != 0) != plus) {
                    Q = plus ? Pc + bit : Pc - bit;   // sibling in the parent's octet
                } else {
                    const int32_t v = T.nbr[(int64_t)dir * T.noct + pog];
                    if (v >= 0) Q = lp.off + 8 * (int64_t)v + (sp ^ bit);
                    else if (v <= -2) bad = 1;        // a refined cell beside a coarser leaf
                }
                int32_t out = -1;
                if (Q >= 0) {
                    const int32_t cq = T.child_oct[Q];
                    if (cq >= 0) out = (int32_t)(cq - l.oct_off);
                    else if (T.cell_flags[Q] & 1) out = (int32_t)(-2 - Q);
                    else bad = 1;
                }
                T.nbr[(int64_t)dir * T.noct + go] = out;
            }
        }
        if (bad) throw std::runtime_error("internal: unbalanced T-junction");
    }
    T.t_oct.clear();
    T.trec.assign(T.noct, -1);
    for (int64_t go = 0; go < T.noct; ++go) {
        bool has_t = false;
        for (int dir = 0; dir < 6; ++dir) has_t |= T.nbr[(int64_t)dir * T.noct + go] <= -2;
        if (has_t) {
            T.trec[go] = (int32_t)T.t_oct.size();
            T.t_oct.push_back((int32_t)go);
        }
    }
    T.nt = (int64_t)T.t_oct.size();

    // ---- canonical faces, grouped by (axis, depth of the finer side) and sorted within a
    // group by the Morton key of the + cell.  The - face of a leaf (same-depth or coarser
    // leaf on its - side) is keyed by the leaf itself, so these come in leaf order; the +
    // face of a fine leaf against a coarser leaf (T record) is keyed by the virtual cell
    // beyond it and is merged in.
    std::vector<int64_t> gcount(3 * (D + 1), 0), gbase(3 * (D + 1) + 1, 0);
    struct MF { int32_t mi, pl; int64_t slot; };
    struct TF { uint64_t key; int32_t mi, pl; int64_t slot; };
    auto leaf_key = [&](int64_t r) -> uint64_t {
        const int d = T.leaf_depth[r];
        if (d == 0) return morton3(T.leaf_i[r], T.leaf_j[r], T.leaf_k[r]);
        const int64_t lc = T.leaf_cell[r] - T.L(d).off;
        return (T.okeys[d - mc][lc >> 3] << 3) | (uint64_t)(lc & 7);
    };
    std::vector<std::vector<MF, NoInitAlloc<MF>>> gm(3 * (D + 1));
    std::vector<std::vector<TF, NoInitAlloc<TF>>> gt(3 * (D + 1));
    // The - face of a leaf on each axis (when the cell beyond it is a leaf) and the + face
    // of a fine leaf against a coarser one, for the three axes in one pass over the leaves
    // of a depth: a counting pass per chunk of leaves, then a writing pass from each chunk's
    // offsets (the lists keep leaf order).
    auto face_of = [&](int64_t r, int a, int64_t off, MF* mf, TF* tf) -> int {
        const int64_t g = T.leaf_cell[r];
        const int s = (int)(g & 7), bit = 1 << a;
        int got = 0;
        int64_t gn = -1;
        if (s & bit) gn = g - bit;
        else {
            const int32_t v = T.nbr[(int64_t)(2 * a) * T.noct + (g >> 3)];
            if (v >= 0) gn = off + 8 * (int64_t)v + (s | bit);
            else if (v <= -2) gn = -2 - (int64_t)v;
        }
        if (gn >= 0 && (T.cell_flags[gn] & 1)) {
            if (mf) *mf = MF{T.cell_rank[gn], (int32_t)r, (int64_t)a * T.ncell + g};
            got |= 1;
        }
        if (s & bit) {
            const int32_t v = T.nbr[(int64_t)(2 * a + 1) * T.noct + (g >> 3)];
            if (v <= -2) {
                if (tf) {
                    int64_t c[3] = {T.leaf_i[r], T.leaf_j[r], T.leaf_k[r]};
                    c[a] += 1;
                    const int32_t t = T.trec[g >> 3];
                    *tf = TF{morton3(c[0], c[1], c[2]), (int32_t)r, T.cell_rank[-2 - (int64_t)v],
                             (int64_t)((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + t};
                }
                got |= 2;
            }
        }
        return got;
    };
#ifdef _OPENMP
    const int nch = std::max(1, omp_get_max_threads() * 8);
#else
    const int nch = 1;
#endif
    for (int d = 0; d <= D; ++d) {
        const int64_t r0 = T.leaf_first[d], n = T.leaf_first[d + 1] - r0;
        const int64_t off = T.L(d).off;
        std::vector<int64_t> cnt((size_t)(nch + 1) * 6, 0);   // [chunk + 1][axis * 2 + list]
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nch; ++c) {
            const int64_t lo = r0 + n * c / nch, hi = r0 + n * (c + 1) / nch;
            int64_t k[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t r = lo; r < hi; ++r)
                for (int a = 0; a < 3; ++a) {
                    const int got = face_of(r, a, off, nullptr, nullptr);
                    k[2 * a] += got & 1;
                    k[2 * a + 1] += got >> 1;
                }
            for (int q = 0; q < 6; ++q) cnt[(size_t)(c + 1) * 6 + q] = k[q];
        }
        for (int c = 0; c < nch; ++c)
            for (int q = 0; q < 6; ++q) cnt[(size_t)(c + 1) * 6 + q] += cnt[(size_t)c * 6 + q];
#pragma omp parallel for schedule(static, 1)
        for (int q = 0; q < 6; ++q) {
            const int gi = (q >> 1) * (D + 1) + d;
            if (q & 1) gt[gi].resize(cnt[(size_t)nch * 6 + q]);
            else gm[gi].resize(cnt[(size_t)nch * 6 + q]);
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nch; ++c) {
            const int64_t lo = r0 + n * c / nch, hi = r0 + n * (c + 1) / nch;
            int64_t k[6];
            for (int q = 0; q < 6; ++q) k[q] = cnt[(size_t)c * 6 + q];
            for (int64_t r = lo; r < hi; ++r)
                for (int a = 0; a < 3; ++a) {
                    MF mf;
                    TF tf;
                    const int got = face_of(r, a, off, &mf, &tf);
                    if (got & 1) gm[a * (D + 1) + d][k[2 * a]++] = mf;
                    if (got & 2) gt[a * (D + 1) + d][k[2 * a + 1]++] = tf;
                }
        }
#pragma omp parallel for schedule(static, 1)
        for (int a = 0; a < 3; ++a) {
            auto& tf = gt[a * (D + 1) + d];
            std::sort(tf.begin(), tf.end(), [](const TF& x, const TF& y) { return x.key < y.key; });
            gcount[a * (D + 1) + d] = (int64_t)(gm[a * (D + 1) + d].size() + tf.size());
        }
    }
    for (size_t q = 0; q < gcount.size(); ++q) gbase[q + 1] = gbase[q] + gcount[q];
    T.nface = gbase.back();
    // (sized without initialisation: the merge below writes every entry, in parallel)
#pragma omp parallel sections
    {
#pragma omp section
        T.f_axis.resize(T.nface);
#pragma omp section
        T.f_depth.resize(T.nface);
#pragma omp section
        T.f_minus.resize(T.nface);
#pragma omp section
        T.f_plus.resize(T.nface);
#pragma omp section
        T.f_slot.resize(T.nface);
#pragma omp section
        T.f_kind.resize(T.nface);
    }
    // Merge each group's two key-ordered lists (no key is in both: a T face's key is a cell
    // that is not a leaf of that depth) in chunks of about 2^20 - faces: chunk c takes the
    // - faces [x_c, x_c+1) and the T faces whose keys fall before the key of - face x_c+1,
    // and writes from position x_c + y_c of its group, as the one-pass merge would.
    struct Chunk { int gi; int64_t x0, x1, y0, y1; };
    std::vector<Chunk> chunks;
    for (int gi = 0; gi < (int)gm.size(); ++gi) {
        const auto& mf = gm[gi];
        const auto& tf = gt[gi];
        const int64_t nx = (int64_t)mf.size(), nc = std::max<int64_t>(1, nx >> 20);
        auto ysplit = [&](int64_t x) -> int64_t {
            const uint64_t key = leaf_key(mf[x].pl);
            return std::lower_bound(tf.begin(), tf.end(), key,
                                    [](const TF& t, uint64_t k) { return t.key < k; }) - tf.begin();
        };
        int64_t x0 = 0, y0 = 0;
        for (int64_t c = 1; c <= nc; ++c) {
            const int64_t x1 = c == nc ? nx : nx * c / nc;
            const int64_t y1 = c == nc ? (int64_t)tf.size() : ysplit(x1);
            chunks.push_back(Chunk{gi, x0, x1, y0, y1});
            x0 = x1;
            y0 = y1;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ci = 0; ci < (int64_t)chunks.size(); ++ci) {
        const Chunk& K = chunks[ci];
        const auto& mf = gm[K.gi];
        const auto& tf = gt[K.gi];
        const int a = K.gi / (D + 1), d = K.gi % (D + 1);
        int64_t f = gbase[K.gi] + K.x0 + K.y0, x = K.x0, y = K.y0;
        while (x < K.x1 || y < K.y1) {
            const bool take_t = y < K.y1 && (x >= K.x1 || tf[y].key < leaf_key(mf[x].pl));
            if (take_t) {
                T.f_minus[f] = tf[y].mi; T.f_plus[f] = tf[y].pl; T.f_slot[f] = tf[y].slot; T.f_kind[f] = 1;
                ++y;
            } else {
                T.f_minus[f] = mf[x].mi; T.f_plus[f] = mf[x].pl; T.f_slot[f] = mf[x].slot; T.f_kind[f] = 0;
                ++x;
            }
            T.f_axis[f] = (int8_t)a;
            T.f_depth[f] = (int8_t)d;
            ++f;
        }
    }
}

void face_plus_cell(const HostTree& T, int64_t f, int32_t& i, int32_t& j, int32_t& k) {
    if (T.f_kind[f] == 0) {
        const int64_t r = T.f_plus[f];
        i = T.leaf_i[r]; j = T.leaf_j[r]; k = T.leaf_k[r];
    } else {
        const int64_t r = T.f_minus[f];
        i = T.leaf_i[r] + (T.f_axis[f] == 0);
        j = T.leaf_j[r] + (T.f_axis[f] == 1);
        k = T.leaf_k[r] + (T.f_axis[f] == 2);
    }
}

void leaf_neighbour(const HostTree& T, int64_t r, int dir, int8_t& kind, int64_t& rank) {
    const int d = T.leaf_depth[r];
    const int64_t g = T.leaf_cell[r];
    const int a = dir >> 1, bit = 1 << a, s = (int)(g & 7);
    const bool plus = dir & 1;
    int64_t gn = -1;
    kind = 0;
    rank = -1;
    if (((s & bit) != 0) != plus) {
        gn = plus ? g + bit : g - bit;
    } else {
        const int32_t v = T.nbr[(int64_t)dir * T.noct + (g >> 3)];
        if (v >= 0) gn = T.L(d).off + 8 * (int64_t)v + (s ^ bit);
        else if (v <= -2) {
            kind = 2;
            rank = T.cell_rank[-2 - (int64_t)v];
            return;
        }
    }
    if (gn < 0) return;
    if (T.cell_flags[gn] & 1) { kind = 1; rank = T.cell_rank[gn]; }
    else kind = 3;
}

// ---------------------------------------------------------------- adjoint tables
void build_adjoint_topology(const HostTree& T, AdjointTopology& out) {
    out = AdjointTopology{};
    // coarse leaves of the T-junctions: the K of every T face of every T octet
    std::vector<int32_t> ks = par_compact<int32_t>(T.nt * 6, [&](int64_t q, int32_t& v) {
        const int64_t go = T.t_oct[q / 6];
        const int32_t n = T.nbr[(q % 6) * T.noct + go];
        v = -2 - n;
        return n <= -2;
    });
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    out.tcoarse = std::move(ks);
    // every octet that is a T octet (the children of a T parent) or lies below one, each
    // listed once: marked top-down level by level (a T octet may itself lie under another
    // T parent), then collected in global octet order
    std::vector<uint8_t> mark(T.noct, 0);
    for (int m = 1; m <= T.D; ++m) {
        const LevelMeta& l = T.L(m);
#pragma omp parallel for schedule(static)
        for (int64_t o = 0; o < l.noct; ++o) {
            const int64_t go = l.oct_off + o;
            mark[go] = (T.trec[go] >= 0 || mark[T.oct_parent[go] >> 3]) ? 1 : 0;
        }
    }
    out.tdesc = par_compact<int32_t>(T.noct, [&](int64_t go, int32_t& v) {
        v = (int32_t)go;
        return mark[go] != 0;
    });
}

}  // namespace ocg
