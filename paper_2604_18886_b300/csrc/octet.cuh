// Level kernels with one thread per octet (sm_103a).
//
// An octet (the 8 children of one coarser cell, slot s = dx + 2 dy + 4 dz) is 8
// consecutive cells, so a thread loads its values and coefficients with 128-bit loads
// and evaluates all 8 stencils in registers: the face between slots s and s ^ (1 << a)
// is internal, and each of the 6 octet faces touches 4 cells of the neighbouring octet
// (table nbr) or, at a T-junction, a coarser leaf K (Sec. 3.1): the ghost
// g = u + (u_K - ubar)/2 uses the mean ubar of this octet's active cells, which the
// thread already holds.  Every kernel here reads the state at launch and writes only
// cells that no other thread of the same launch reads (sweeps write the cells of one
// colour, whose face neighbours are all of the other colour).
#pragma once

#include "kernels.cuh"

namespace ocg {

constexpr int OBLK = 64;   // threads (octets) per block: spreads small levels over all SMs

// slots with bit a clear, in the order of the T-record sub-face index q
__device__ __forceinline__ int clear_slot(int a, int q) {
    return a == 0 ? 2 * q : (a == 1 ? ((q & 1) | ((q & 2) << 1)) : q);
}

__device__ __forceinline__ void ld8(const float* __restrict__ p, float (&r)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
__device__ __forceinline__ void ld8(const double* __restrict__ p, double (&r)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double2 a = reinterpret_cast<const double2*>(p)[q];
        r[2 * q] = a.x;
        r[2 * q + 1] = a.y;
    }
}
__device__ __forceinline__ void st8(float* __restrict__ p, const float (&r)[8]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(r[0], r[1], r[2], r[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(r[4], r[5], r[6], r[7]);
}
__device__ __forceinline__ void st8(double* __restrict__ p, const double (&r)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(r[2 * q], r[2 * q + 1]);
}
// read-only coefficient loads, converted to the arithmetic type
__device__ __forceinline__ void ldc8(const float* __restrict__ p, float (&r)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
__device__ __forceinline__ void ldc8(const float* __restrict__ p, double (&r)[8]) {
    float t[8];
    ldc8(p, t);
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = t[q];
}
__device__ __forceinline__ void ldc8(const double* __restrict__ p, double (&r)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p) + q);
        r[2 * q] = a.x;
        r[2 * q + 1] = a.y;
    }
}
__device__ __forceinline__ void ldc8(const double* __restrict__ p, float (&r)[8]) {
    double t[8];
    ldc8(p, t);
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = (float)t[q];
}
__device__ __forceinline__ void ldc8(const __nv_bfloat16* __restrict__ p, float (&r)[8]) {
    const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h[q]);
        r[2 * q] = f.x;
        r[2 * q + 1] = f.y;
    }
}

// The four cells of the octet at p on one side of axis a (the cells whose bit a equals
// side), in the sub-face order q of clear_slot.  A z layer is four consecutive cells and a
// y layer two pairs, so both come in vector loads (one request per 16 or 8 bytes instead
// of one per cell); an x layer is every other cell.  p is the octet's first cell, so 16-byte
// aligned for 4-byte types.  The values are the ones the per-cell loads would return.
template <class T>
__device__ __forceinline__ T ld1(const T* p, bool ro) { return ro ? __ldg(p) : *p; }
template <class V>
__device__ __forceinline__ V ldv(const void* p, bool ro) {
    return ro ? __ldg(reinterpret_cast<const V*>(p)) : *reinterpret_cast<const V*>(p);
}
__device__ __forceinline__ void ld_layer(const float* __restrict__ p, int a, int side, bool ro, float (&r)[4]) {
    if (a == 2) {
        const float4 v = ldv<float4>(p + 4 * side, ro);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if (a == 1) {
        const float2 v0 = ldv<float2>(p + 2 * side, ro), v1 = ldv<float2>(p + 4 + 2 * side, ro);
        r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = ld1(p + 2 * q + side, ro);
    }
}
__device__ __forceinline__ void ld_layer(const double* __restrict__ p, int a, int side, bool ro, double (&r)[4]) {
    if (a == 2) {
        const double2 v0 = ldv<double2>(p + 4 * side, ro), v1 = ldv<double2>(p + 4 * side + 2, ro);
        r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
    } else if (a == 1) {
        const double2 v0 = ldv<double2>(p + 2 * side, ro), v1 = ldv<double2>(p + 4 + 2 * side, ro);
        r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = ld1(p + 2 * q + side, ro);
    }
}
__device__ __forceinline__ void ld_layer(const __nv_bfloat16* __restrict__ p, int a, int side, bool ro,
                                         __nv_bfloat16 (&r)[4]) {
    if (a == 2) {
        const uint2 v = ldv<uint2>(p + 4 * side, ro);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = h[q];
    } else if (a == 1) {
        const __nv_bfloat162 v0 = ldv<__nv_bfloat162>(p + 2 * side, ro), v1 = ldv<__nv_bfloat162>(p + 4 + 2 * side, ro);
        r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = ld1(p + 2 * q + side, ro);
    }
}

// ------------------------------------------------ vectors in either layout (CY: cycle)
// One colour chunk (the 4 cells of colour col of the octet at c8, in the colour's slot
// order k = s >> 1) of a vector in the cycle layout.
__device__ __forceinline__ void ldk4(const float* __restrict__ U, int c8, int col, float (&r)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(U + cyc8(c8) + 32 * col);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
}
__device__ __forceinline__ void ldk4(const double* __restrict__ U, int c8, int col, double (&r)[4]) {
    const double2* p = reinterpret_cast<const double2*>(U + cyc8(c8) + 32 * col);
    const double2 a = p[0], b = p[1];
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}
__device__ __forceinline__ void stk4(float* __restrict__ U, int c8, int col, const float (&r)[4]) {
    *reinterpret_cast<float4*>(U + cyc8(c8) + 32 * col) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void stk4(double* __restrict__ U, int c8, int col, const double (&r)[4]) {
    double2* p = reinterpret_cast<double2*>(U + cyc8(c8) + 32 * col);
    p[0] = make_double2(r[0], r[1]);
    p[1] = make_double2(r[2], r[3]);
}
// slot of the k-th cell of colour col
__host__ __device__ __forceinline__ constexpr int colour_slot(int col, int k) {
    return 2 * k + (((k ^ (k >> 1)) & 1) ^ col);
}
// the 8 values of the octet at c8 in slot order, from either layout
template <bool CY, class TV>
__device__ __forceinline__ void ldv8(const TV* __restrict__ U, int c8, TV (&r)[8]) {
    if (CY) {
        TV k0[4], k1[4];
        ldk4(U, c8, 0, k0);
        ldk4(U, c8, 1, k1);
#pragma unroll
        for (int k = 0; k < 4; ++k) { r[colour_slot(0, k)] = k0[k]; r[colour_slot(1, k)] = k1[k]; }
    } else {
        ld8(U + c8, r);
    }
}
template <bool CY, class TV>
__device__ __forceinline__ void stv8(TV* __restrict__ U, int c8, const TV (&r)[8]) {
    if (CY) {
        TV k0[4], k1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { k0[k] = r[colour_slot(0, k)]; k1[k] = r[colour_slot(1, k)]; }
        stk4(U, c8, 0, k0);
        stk4(U, c8, 1, k1);
    } else {
        st8(U + c8, r);
    }
}
// the four cells of the octet at n8 with bit a equal to side, in sub-face order q (as
// ld_layer), from either layout
template <bool CY, class TV>
__device__ __forceinline__ void ldv_layer(const TV* __restrict__ U, int n8, int a, int side, TV (&r)[4]) {
    if (CY) {
        TV v[8];
        ldv8<true>(U, n8, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = v[clear_slot(a, q) | (side << a)];
    } else {
        ld_layer(U + n8, a, side, false, r);
    }
}

// Coordinates of octet o in a lexicographic ni^3 grid (shifts when ni is a power of two).
__device__ __forceinline__ void octet_coords(int o, int ni, int& I, int& J, int& K) {
    if ((ni & (ni - 1)) == 0) {
        const int sh = __ffs(ni) - 1;
        I = o & (ni - 1);
        J = (o >> sh) & (ni - 1);
        K = o >> (2 * sh);
    } else {
        I = o % ni;
        J = (o / ni) % ni;
        K = o / (ni * ni);
    }
}

// 1/n for the mean of n active cells (n <= 8): multiply instead of divide; 0 for n = 0, so
// that the mean over no active cell is 0 (Alg. 3's active count; inactive cells have no
// coefficient, and an infinite factor would turn their zero terms into NaN)
template <class TV>
__device__ __forceinline__ TV inv_count(int n) {
    return n == 8 ? TV(0.125)
                  : (n == 4 ? TV(0.25) : (n == 2 ? TV(0.5) : (n == 1 ? TV(1) : (n == 0 ? TV(0) : TV(1) / TV(n)))));
}

template <class TV>
struct OctState {
    TV u[8], d[8], cm[3][8];
    TV ubar;      // mean of the active cells
    int nact;
};

// Loads u (plain or cycle layout, CY) and the coefficients of the octet whose first cell
// is c8.
template <class TV, class TC, class TW, bool CY = false>
__device__ __forceinline__ void load_octet(const TV* __restrict__ U, const Coefs<TC, TW>& C, int c8,
                                           OctState<TV>& S) {
    ldv8<CY>(U, c8, S.u);
    ldc8(C.d + c8, S.d);
    ldc8(C.cx + c8, S.cm[0]);
    ldc8(C.cy + c8, S.cm[1]);
    ldc8(C.cz + c8, S.cm[2]);
}

template <class TV>
__device__ __forceinline__ void octet_mean(OctState<TV>& S) {
    TV s = TV(0);
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (S.d[q] != TV(0)) { s += S.u[q]; ++n; }
    S.nact = n;
    S.ubar = s * inv_count<TV>(n);
}

// The six neighbouring octets of local octet o: on a uniform level (ni > 0, octets in
// lexicographic order) computed from o, otherwise read from the table (values: local
// octet, -1 wall, -2-K for a face covered by the coarser leaf K).
__device__ __forceinline__ void octet_neighbours(const Tables& T, int ni, int o, int og, int (&nb)[6]) {
    if (ni > 0) {
        int I, J, K;
        octet_coords(o, ni, I, J, K);
        const int sy = ni, sz = ni * ni;
        nb[0] = I > 0 ? o - 1 : -1;
        nb[1] = I < ni - 1 ? o + 1 : -1;
        nb[2] = J > 0 ? o - sy : -1;
        nb[3] = J < ni - 1 ? o + sy : -1;
        nb[4] = K > 0 ? o - sz : -1;
        nb[5] = K < ni - 1 ? o + sz : -1;
    } else {
#pragma unroll
        for (int dir = 0; dir < 6; ++dir) nb[dir] = __ldg(T.nbr + dir * T.noct + og);
    }
}

// neighbouring octet of local octet o in direction dir (arithmetic on uniform levels)
__device__ __forceinline__ int octet_neighbour(const Tables& T, int ni, int o, int og, int dir) {
    if (ni > 0) {
        int c[3];
        octet_coords(o, ni, c[0], c[1], c[2]);
        const int a = dir >> 1;
        const int stride = a == 0 ? 1 : (a == 1 ? ni : ni * ni);
        if (dir & 1) return c[a] < ni - 1 ? o + stride : -1;
        return c[a] > 0 ? o - stride : -1;
    }
    return __ldg(T.nbr + dir * T.noct + og);
}

template <class T>
__device__ __forceinline__ T divide(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float divide<float>(float a, float b) { return __fdividef(a, b); }

// Au[s] = (A^m u) for the 8 cells of local octet o (global og) of the level A; U (plain or
// cycle layout, CY) is read for the neighbouring octets and the coarser leaves K of T faces.
template <class TV, class TC, class TW, bool CY = false>
__device__ __forceinline__ void octet_Au(const Tables& T, const Coefs<TC, TW>& C, const TV* __restrict__ U,
                                         const LevelArgs& A, int o, int og, const OctState<TV>& S, TV (&Au)[8]) {
#pragma unroll
    for (int s = 0; s < 8; ++s) Au[s] = S.d[s] * S.u[s];
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    const int off = A.off;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        // internal faces (s, s | bit), coefficient kept by the + cell
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), t = s | bit;
            const TV c = S.cm[a][t];
            Au[s] += c * S.u[t];
            Au[t] += c * S.u[s];
        }
        // - face: cells with bit clear meet the + side of the - neighbour
        const int v = nb[2 * a];
        if (v >= 0) {
            const int n8 = off + 8 * v;
            TV nu[4];
            ldv_layer<CY>(U, n8, a, 1, nu);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += S.cm[a][s] * nu[q];
            }
        } else if (v <= -2) {
            const TV uK = U[vidx<CY>(-2 - v)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += S.cm[a][s] * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
        // + face: cells with bit set meet the - side of the + neighbour, whose cells keep
        // the face coefficients; at a T face the fine coefficients are in the T record
        const int w = nb[2 * a + 1];
        if (w >= 0) {
            const int n8 = off + 8 * w;
            const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
            TV nu[4], nc[4];
            TC ncr[4];
            ldv_layer<CY>(U, n8, a, 0, nu);
            ld_layer(cc + n8, a, 0, true, ncr);
#pragma unroll
            for (int q = 0; q < 4; ++q) nc[q] = TV(tov(ncr[q]));
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[clear_slot(a, q) | bit] += nc[q] * nu[q];
        } else if (w <= -2) {
            const TV uK = U[vidx<CY>(-2 - w)];
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit;
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + q) * T.nt + t)));
                Au[s] += cf * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
    }
}

// u of the children octet co += uP - (mean of its active cells); U in the cycle layout
// (both colour chunks rewritten, the inactive cells unchanged: one thread owns the octet)
template <class TV, class TC>
__device__ __forceinline__ void octet_prolong(const TC* __restrict__ d, TV* __restrict__ U, int co, TV uP) {
    const int c8 = 8 * co;
    TV v[8], dd[8];
    ldv8<true>(U, c8, v);
    ldc8(d + c8, dd);
    TV s = TV(0);
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != TV(0)) { s += v[q]; ++n; }
    if (n == 0) return;
    const TV delta = uP - s * inv_count<TV>(n);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != TV(0)) v[q] = v[q] + delta;
    stv8<true>(U, c8, v);
}

// Completion of the FAS right-hand side b += A^m u* on the cells with children of a level
// (Alg. 4); u and b in the cycle layout.
template <class TV, class TC, class TW>
__device__ __forceinline__ void ofixb_octet(const LevelArgs& A, const Tables& T, const Coefs<TC, TW>& C,
                                            const TV* __restrict__ U, TV* __restrict__ B, int o) {
    const int c8 = A.off + 8 * o;
    const int og = c8 >> 3;
    OctState<TV> S;
    load_octet<TV, TC, TW, true>(U, C, c8, S);
    octet_mean(S);
    TV b[8], Au[8];
    ldv8<true>(B, c8, b);
    octet_Au<TV, TC, TW, true>(T, C, U, A, o, og, S, Au);
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (__ldg(T.child_oct + c8 + s) >= 0) b[s] = b[s] + Au[s];
    stv8<true>(B, c8, b);
}

// Red-black colour sweep (Sec. 2.3) of a level, colour COL: u += (b - A^m u) / c on the
// 4 cells of colour COL of octet o, every read from the state at launch.  Only the rows
// of the colour are formed (the terms of each row summed in the order of octet_Au); from
// each neighbouring octet only its other-colour chunk is read, which holds the 2 cells
// facing this octet's cells of colour COL; b is read and u written as one chunk each.
// prolong: after the update, every cell with children prolongs its final value onto them.
template <class TV, class TC, class TW, int COL>
__device__ __forceinline__ void osweep_colour(const LevelArgs& A, const Tables& T, const Coefs<TC, TW>& C,
                                              TV* __restrict__ U, const TV* __restrict__ B, int o, int prolong) {
    const int c8 = A.off + 8 * o;
    const int og = c8 >> 3;
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    OctState<TV> S;
    load_octet<TV, TC, TW, true>(U, C, c8, S);
    TV b[4];
    ldk4(B, c8, COL, b);
    octet_mean(S);
    const int off = A.off;
    TV Au[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int s = colour_slot(COL, k);
        Au[k] = S.d[s] * S.u[s];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const int v = nb[2 * a], w = nb[2 * a + 1];
        TV vu[4], wu[4];
        if (v >= 0) ldk4(U, off + 8 * v, 1 - COL, vu);
        if (w >= 0) ldk4(U, off + 8 * w, 1 - COL, wu);
        const TV uKv = v <= -2 ? U[cyc(-2 - v)] : TV(0);
        const TV uKw = w <= -2 ? U[cyc(-2 - w)] : TV(0);
        const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = colour_slot(COL, k), t = s ^ bit;
            // internal face (s, t), coefficient kept by the + cell
            Au[k] += ((s & bit) ? S.cm[a][s] : S.cm[a][t]) * S.u[t];
            if (!(s & bit)) {
                // - face: the - neighbour's cell s | bit (other colour, chunk slot t >> 1)
                if (v >= 0) Au[k] += S.cm[a][s] * vu[t >> 1];
                else if (v <= -2) Au[k] += S.cm[a][s] * (S.u[s] + (uKv - S.ubar) * TV(0.5));
            } else {
                // + face: the + neighbour's cell t = s & ~bit keeps the face coefficient; at a
                // T face the fine weight is in the T record
                if (w >= 0) Au[k] += TV(tov(__ldg(cc + off + 8 * w + t))) * wu[t >> 1];
                else if (w <= -2) {
                    const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + sub_index(a, t)) * T.nt + __ldg(T.trec + og))));
                    Au[k] += cf * (S.u[s] + (uKw - S.ubar) * TV(0.5));
                }
            }
        }
    }
    TV un[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int s = colour_slot(COL, k);
        un[k] = S.d[s] != TV(0) ? S.u[s] + divide(b[k] - Au[k], S.d[s]) : S.u[s];
    }
    stk4(U, c8, COL, un);
    if (prolong) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int co = __ldg(T.child_oct + c8 + s);
            if (co >= 0) octet_prolong<TV>(C.d, U, co, cyc_colour(s) == COL ? un[s >> 1] : S.u[s]);
        }
    }
}

// Either colour sweep (colour at run time) or, with fixb, the FAS right-hand-side pass.
template <class TV, class TC, class TW>
__device__ __forceinline__ void osweep_octet(const LevelArgs& A, const Tables& T, const Coefs<TC, TW>& C,
                                             TV* __restrict__ U, TV* __restrict__ B, int o, int colour,
                                             int prolong, int fixb) {
    if (fixb) ofixb_octet<TV, TC, TW>(A, T, C, U, B, o);
    else if (colour) osweep_colour<TV, TC, TW, 1>(A, T, C, U, B, o, prolong);
    else osweep_colour<TV, TC, TW, 0>(A, T, C, U, B, o, prolong);
}

// MODE 0 / 1: colour sweep of that colour; 2: the FAS right-hand-side pass
template <class TV, class TC, class TW, int MODE>
__global__ void __launch_bounds__(OBLK, sizeof(TV) == 4 ? 16 : 8) k_osweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                 TV* __restrict__ B, int prolong) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    if (MODE == 2) ofixb_octet<TV, TC, TW>(A, T, C, U, B, o);
    else osweep_colour<TV, TC, TW, MODE>(A, T, C, U, B, o, prolong);
}

// ------------------------------------------------------------ shared-block sweep
// The octet form with the block's u and face coefficients shared: each thread loads its
// octet (as in k_osweep) and also places u, c_x-, c_y-, c_z- in shared memory, slot-major
// (index s * TBLK + local octet, conflict-free across a warp); reads of a neighbouring
// octet that lies in the same block (most of them on Morton-ordered levels) then come
// from shared memory instead of a scattered global load.
constexpr int TBLK = 128;

template <class TV>
struct TileSh {
    TV u[8 * TBLK], cm[3][8 * TBLK];
};

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(TBLK) k_tsweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                 TV* __restrict__ B, int colour, int prolong) {
    pdl_enter();
    __shared__ TileSh<TV> sh;
    const int noct = A.ncell >> 3;
    const int o0 = blockIdx.x * TBLK, lo = threadIdx.x;
    const int o = o0 + lo;
    const bool valid = o < noct;
    const int c8 = A.off + 8 * (valid ? o : noct - 1), og = c8 >> 3;
    // the neighbour indices are loaded with the octet, before the barrier
    int nb[6];
    octet_neighbours(T, A.ni, valid ? o : noct - 1, og, nb);
    OctState<TV> S;
    load_octet<TV, TC, TW, true>(U, C, c8, S);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        sh.u[q * TBLK + lo] = S.u[q];
        sh.cm[0][q * TBLK + lo] = S.cm[0][q];
        sh.cm[1][q * TBLK + lo] = S.cm[1][q];
        sh.cm[2][q * TBLK + lo] = S.cm[2][q];
    }
    __syncthreads();
    if (!valid) return;
    octet_mean(S);
    TV b[8], Au[8];
    ldv8<true>(B, c8, b);
#pragma unroll
    for (int q = 0; q < 8; ++q) Au[q] = S.d[q] * S.u[q];
    const int off = A.off;
    const int nend = min(TBLK, noct - o0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), t = s | bit;
            const TV c = S.cm[a][t];
            Au[s] += c * S.u[t];
            Au[t] += c * S.u[s];
        }
        const int v = nb[2 * a];
        if (v >= 0) {
            const int lv = v - o0;
            TV nu[4];
            if (lv >= 0 && lv < nend) {
#pragma unroll
                for (int q = 0; q < 4; ++q) nu[q] = sh.u[(clear_slot(a, q) | bit) * TBLK + lv];
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) nu[q] = U[cyc(off + 8 * v + (clear_slot(a, q) | bit))];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[clear_slot(a, q)] += S.cm[a][clear_slot(a, q)] * nu[q];
        } else if (v <= -2) {
            const TV uK = U[cyc(-2 - v)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += S.cm[a][s] * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
        const int w = nb[2 * a + 1];
        if (w >= 0) {
            const int lw = w - o0;
            TV nu[4], nc[4];
            if (lw >= 0 && lw < nend) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    nu[q] = sh.u[clear_slot(a, q) * TBLK + lw];
                    nc[q] = sh.cm[a][clear_slot(a, q) * TBLK + lw];
                }
            } else {
                const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    nu[q] = U[cyc(off + 8 * w + clear_slot(a, q))];
                    nc[q] = TV(tov(__ldg(cc + off + 8 * w + clear_slot(a, q))));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[clear_slot(a, q) | bit] += nc[q] * nu[q];
        } else if (w <= -2) {
            const TV uK = U[cyc(-2 - w)];
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit;
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + q) * T.nt + t)));
                Au[s] += cf * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
    }
    TV un[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        un[s] = S.u[s];
        if (((__popc(s) & 1) == colour) && S.d[s] != TV(0)) {
            un[s] = S.u[s] + divide(b[s] - Au[s], S.d[s]);
            U[cyc(c8 + s)] = un[s];
        }
    }
    if (prolong) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int co = __ldg(T.child_oct + c8 + s);
            if (co >= 0) octet_prolong<TV>(C.d, U, co, un[s]);
        }
    }
}

// ------------------------------------------------------------ thread-per-cell sweep
// The same colour sweep with one thread per cell: the octet's 8 cells are 8 consecutive
// lanes, in-octet neighbours and the T-ghost sibling mean come from warp shuffles, the
// neighbour across the octet boundary from the neighbour octet (arithmetic on uniform
// levels, table on adaptive ones).  Shorter per-thread dependency chains and 8x more
// warps than k_osweep; the autotuner picks the faster form per level.
template <class T>
__device__ __forceinline__ T lane_octet_sum(T v) {
    v += __shfl_xor_sync(FULL, v, 1);
    v += __shfl_xor_sync(FULL, v, 2);
    v += __shfl_xor_sync(FULL, v, 4);
    return v;
}

// tid: thread index within the level (the 8 lanes of an octet are consecutive and
// aligned to 8 inside the warp); threads past the level's end work on a copy of the last
// octet so that the warp shuffles stay full, and write nothing.
template <class TV, class TC, class TW>
__device__ __forceinline__ void csweep_cell(const LevelArgs& A, const Tables& T, const Coefs<TC, TW>& C,
                                            TV* __restrict__ U, TV* __restrict__ B, int tid, int colour,
                                            int prolong) {
    const bool valid = tid < A.ncell;
    const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int g = A.off + lc;
    const int s = lc & 7, o = lc >> 3, og = g >> 3;
    const TV u = U[cyc(g)];
    const TV b = B[cyc(g)];
    const TV dd = TV(tov(__ldg(C.d + g)));
    const TV cm[3] = {TV(tov(__ldg(C.cx + g))), TV(tov(__ldg(C.cy + g))), TV(tov(__ldg(C.cz + g)))};
    const bool act = dd != TV(0);
    // outer neighbour octet per axis: the + octet if bit a of s is set, else the - octet
    int nbo[3];
    if (A.ni > 0) {
        int crd[3];
        octet_coords(o, A.ni, crd[0], crd[1], crd[2]);
        const int stride[3] = {1, A.ni, A.ni * A.ni};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            nbo[a] = (s >> a) & 1 ? (crd[a] < A.ni - 1 ? o + stride[a] : -1) : (crd[a] > 0 ? o - stride[a] : -1);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) nbo[a] = __ldg(T.nbr + (2 * a + ((s >> a) & 1)) * T.noct + og);
    }
    const TV us = lane_octet_sum<TV>(act ? u : TV(0));
    const unsigned bal = __ballot_sync(FULL, act);
    const int cnt = __popc((bal >> (threadIdx.x & 24)) & 0xffu);
    const TV ubar = us * inv_count<TV>(cnt);
    TV Au = dd * u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const TV u_in = __shfl_xor_sync(FULL, u, bit);
        const TV c_in = __shfl_xor_sync(FULL, cm[a], bit);
        const int v = nbo[a];
        if (s & bit) {
            Au += cm[a] * u_in;
            if (v >= 0) {
                const int ng = A.off + 8 * v + (s ^ bit);
                const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
                Au += TV(tov(__ldg(cc + ng))) * U[cyc(ng)];
            } else if (v <= -2) {
                const int t = __ldg(T.trec + og);
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + t)));
                Au += cf * (u + (U[cyc(-2 - v)] - ubar) * TV(0.5));
            }
        } else {
            Au += c_in * u_in;
            if (v >= 0) Au += cm[a] * U[cyc(A.off + 8 * v + (s ^ bit))];
            else if (v <= -2) Au += cm[a] * (u + (U[cyc(-2 - v)] - ubar) * TV(0.5));
        }
    }
    TV un = u;
    if (valid && act && ((__popc(s) & 1) == colour)) {
        un = u + divide(b - Au, dd);
        U[cyc(g)] = un;
    }
    if (prolong && valid) {
        const int co = __ldg(T.child_oct + g);
        if (co >= 0) octet_prolong<TV>(C.d, U, co, un);
    }
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_csweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                TV* __restrict__ B, int colour, int prolong) {
    pdl_enter();
    csweep_cell<TV, TC, TW>(A, T, C, U, B, blockIdx.x * BLK + threadIdx.x, colour, prolong);
}

// ------------------------------------------------------------ half-octet sweep
// The same colour sweep with two threads per octet: thread hz = lane & 1 owns the z-layer
// hz (slots 4 hz .. 4 hz + 3, contiguous), so its values and coefficients arrive in one
// vector load per array (16 B in FP32); the partner lane (lane ^ 1) holds the other layer
// and supplies the z-neighbours inside the octet and its half of the T-ghost mean by
// shuffles; the face to a neighbouring octet reads that octet's matching layer with one
// vector load (x and y faces: the same layer; z faces: the facing layer).  In-layer index
// q = dx + 2 dy.
__device__ __forceinline__ void ld4(const float* __restrict__ p, float (&r)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* __restrict__ p, double (&r)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}
__device__ __forceinline__ void st4(float* __restrict__ p, const float (&r)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double* __restrict__ p, const double (&r)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(r[2], r[3]);
}
template <class TV>
__device__ __forceinline__ void ldc4(const float* __restrict__ p, TV (&r)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = TV(a.x); r[1] = TV(a.y); r[2] = TV(a.z); r[3] = TV(a.w);
}
template <class TV>
__device__ __forceinline__ void ldc4(const double* __restrict__ p, TV (&r)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    r[0] = TV(a.x); r[1] = TV(a.y); r[2] = TV(b.x); r[3] = TV(b.y);
}
template <class TV>
__device__ __forceinline__ void ldc4(const __nv_bfloat16* __restrict__ p, TV (&r)[4]) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
    const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
    r[0] = TV(f0.x); r[1] = TV(f0.y); r[2] = TV(f1.x); r[3] = TV(f1.y);
}

// z layer hz (slots 4 hz .. 4 hz + 3, in that order) of the octet at c8 of a vector in the
// cycle layout: two pairs, ranks 2 hz and 2 hz + 1 of each colour chunk (layer 0: slots 0, 3
// of colour 0 and 1, 2 of colour 1; layer 1: slots 5, 6 and 4, 7).
__device__ __forceinline__ void ldh4(const float* __restrict__ U, int c8, int hz, float (&r)[4]) {
    const float2 v0 = *reinterpret_cast<const float2*>(U + cyc8(c8) + 2 * hz);
    const float2 v1 = *reinterpret_cast<const float2*>(U + cyc8(c8) + 32 + 2 * hz);
    r[0] = hz ? v1.x : v0.x; r[1] = hz ? v0.x : v1.x; r[2] = hz ? v0.y : v1.y; r[3] = hz ? v1.y : v0.y;
}
__device__ __forceinline__ void ldh4(const double* __restrict__ U, int c8, int hz, double (&r)[4]) {
    const double2 v0 = *reinterpret_cast<const double2*>(U + cyc8(c8) + 2 * hz);
    const double2 v1 = *reinterpret_cast<const double2*>(U + cyc8(c8) + 32 + 2 * hz);
    r[0] = hz ? v1.x : v0.x; r[1] = hz ? v0.x : v1.x; r[2] = hz ? v0.y : v1.y; r[3] = hz ? v1.y : v0.y;
}
__device__ __forceinline__ void sth4(float* __restrict__ U, int c8, int hz, const float (&r)[4]) {
    *reinterpret_cast<float2*>(U + cyc8(c8) + 2 * hz) = hz ? make_float2(r[1], r[2]) : make_float2(r[0], r[3]);
    *reinterpret_cast<float2*>(U + cyc8(c8) + 32 + 2 * hz) = hz ? make_float2(r[0], r[3]) : make_float2(r[1], r[2]);
}
__device__ __forceinline__ void sth4(double* __restrict__ U, int c8, int hz, const double (&r)[4]) {
    *reinterpret_cast<double2*>(U + cyc8(c8) + 2 * hz) = hz ? make_double2(r[1], r[2]) : make_double2(r[0], r[3]);
    *reinterpret_cast<double2*>(U + cyc8(c8) + 32 + 2 * hz) = hz ? make_double2(r[0], r[3]) : make_double2(r[1], r[2]);
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_qsweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                TV* __restrict__ B, int colour, int prolong) {
    pdl_enter();
    const int tid = blockIdx.x * BLK + threadIdx.x;
    const int noct = A.ncell >> 3;
    const bool valid = (tid >> 1) < noct;
    const int o = valid ? (tid >> 1) : noct - 1;   // past the end: a copy of the last octet, no writes
    const int hz = tid & 1;
    const int c8 = A.off + 8 * o, og = c8 >> 3, base = c8 + 4 * hz;
    TV u[4], b[4], d[4], cx[4], cy[4], cz[4];
    ldh4(U, c8, hz, u);
    ldh4(B, c8, hz, b);
    ldc4<TV>(C.d + base, d);
    ldc4<TV>(C.cx + base, cx);
    ldc4<TV>(C.cy + base, cy);
    ldc4<TV>(C.cz + base, cz);
    // octet mean over the active cells (both layers)
    TV ssum = TV(0);
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (d[q] != TV(0)) { ssum += u[q]; ++cnt; }
    ssum += __shfl_xor_sync(FULL, ssum, 1);
    cnt += __shfl_xor_sync(FULL, cnt, 1);
    const TV ubar = ssum * inv_count<TV>(cnt);
    TV up[4], czp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        up[q] = __shfl_xor_sync(FULL, u[q], 1);
        czp[q] = __shfl_xor_sync(FULL, cz[q], 1);
    }
    TV Au[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Au[q] = d[q] * u[q];
    // faces inside the layer (coefficient kept by the + cell) and between the layers
    Au[0] += cx[1] * u[1]; Au[1] += cx[1] * u[0]; Au[2] += cx[3] * u[3]; Au[3] += cx[3] * u[2];
    Au[0] += cy[2] * u[2]; Au[2] += cy[2] * u[0]; Au[1] += cy[3] * u[3]; Au[3] += cy[3] * u[1];
#pragma unroll
    for (int q = 0; q < 4; ++q) Au[q] += (hz ? cz[q] : czp[q]) * up[q];
    const int off = A.off;
    const TV half = TV(0.5);
    // x- : cells q = 0, 2 against the - octet's q = 1, 3 of this layer
    {
        const int v = octet_neighbour(T, A.ni, o, og, 0);
        if (v >= 0) {
            TV nu[4];
            ldh4(U, off + 8 * v, hz, nu);
            Au[0] += cx[0] * nu[1];
            Au[2] += cx[2] * nu[3];
        } else if (v <= -2) {
            const TV uK = U[cyc(-2 - v)];
            Au[0] += cx[0] * (u[0] + (uK - ubar) * half);
            Au[2] += cx[2] * (u[2] + (uK - ubar) * half);
        }
    }
    // y- : cells q = 0, 1 against the - octet's q = 2, 3
    {
        const int v = octet_neighbour(T, A.ni, o, og, 2);
        if (v >= 0) {
            TV nu[4];
            ldh4(U, off + 8 * v, hz, nu);
            Au[0] += cy[0] * nu[2];
            Au[1] += cy[1] * nu[3];
        } else if (v <= -2) {
            const TV uK = U[cyc(-2 - v)];
            Au[0] += cy[0] * (u[0] + (uK - ubar) * half);
            Au[1] += cy[1] * (u[1] + (uK - ubar) * half);
        }
    }
    // x+ : cells q = 1, 3 against the + octet's q = 0, 2 (their c_x- is the face's)
    {
        const int w = octet_neighbour(T, A.ni, o, og, 1);
        if (w >= 0) {
            TV nu[4], nc[4];
            ldh4(U, off + 8 * w, hz, nu);
            ldc4<TV>(C.cx + off + 8 * w + 4 * hz, nc);
            Au[1] += nc[0] * nu[0];
            Au[3] += nc[2] * nu[2];
        } else if (w <= -2) {
            const TV uK = U[cyc(-2 - w)];
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = 2 * k + 1;   // sub-face index of slot 4 hz + q on the x+ face
                const TV cf = TV(tov(__ldg(C.tw + (1 * 4 + (k | (hz << 1))) * T.nt + t)));
                Au[q] += cf * (u[q] + (uK - ubar) * half);
            }
        }
    }
    // y+ : cells q = 2, 3 against the + octet's q = 0, 1
    {
        const int w = octet_neighbour(T, A.ni, o, og, 3);
        if (w >= 0) {
            TV nu[4], nc[4];
            ldh4(U, off + 8 * w, hz, nu);
            ldc4<TV>(C.cy + off + 8 * w + 4 * hz, nc);
            Au[2] += nc[0] * nu[0];
            Au[3] += nc[1] * nu[1];
        } else if (w <= -2) {
            const TV uK = U[cyc(-2 - w)];
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = 2 + k;       // sub-face index (q & 1) | (hz << 1) on the y+ face
                const TV cf = TV(tov(__ldg(C.tw + (3 * 4 + (k | (hz << 1))) * T.nt + t)));
                Au[q] += cf * (u[q] + (uK - ubar) * half);
            }
        }
    }
    // z : layer 0 faces the - octet's layer 1, layer 1 faces the + octet's layer 0
    if (hz == 0) {
        const int v = octet_neighbour(T, A.ni, o, og, 4);
        if (v >= 0) {
            TV nu[4];
            ldh4(U, off + 8 * v, 1, nu);
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[q] += cz[q] * nu[q];
        } else if (v <= -2) {
            const TV uK = U[cyc(-2 - v)];
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[q] += cz[q] * (u[q] + (uK - ubar) * half);
        }
    } else {
        const int w = octet_neighbour(T, A.ni, o, og, 5);
        if (w >= 0) {
            TV nu[4], nc[4];
            ldh4(U, off + 8 * w, 0, nu);
            ldc4<TV>(C.cz + off + 8 * w, nc);
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[q] += nc[q] * nu[q];
        } else if (w <= -2) {
            const TV uK = U[cyc(-2 - w)];
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const TV cf = TV(tov(__ldg(C.tw + (5 * 4 + q) * T.nt + t)));
                Au[q] += cf * (u[q] + (uK - ubar) * half);
            }
        }
    }
    TV un[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int s = 4 * hz + q;
        un[q] = ((__popc(s) & 1) == colour && d[q] != TV(0)) ? u[q] + divide(b[q] - Au[q], d[q]) : u[q];
    }
    if (!valid) return;
    sth4(U, c8, hz, un);   // the other colour's values are rewritten unchanged
    if (prolong) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int co = __ldg(T.child_oct + base + q);
            if (co >= 0) octet_prolong<TV>(C.d, U, co, un[q]);
        }
    }
}

// Residual and FAS restriction (Alg. 4): r = b - A^m u; the parent gets
// b_P = (beta/alpha) sum r (A^{m-1} u* is added on the coarse level by the fixb pass) and
// u_P = u* = mean of the active children.
template <class TV, class TC, class TW>
__device__ __forceinline__ void orestrict_octet(const LevelArgs& A, const Tables& T, const Coefs<TC, TW>& C,
                                                TV* __restrict__ U, TV* __restrict__ B, TV scale, int o) {
    const int c8 = A.off + 8 * o;
    const int og = c8 >> 3;
    OctState<TV> S;
    load_octet<TV, TC, TW, true>(U, C, c8, S);
    octet_mean(S);
    TV b[8], Au[8];
    ldv8<true>(B, c8, b);
    octet_Au<TV, TC, TW, true>(T, C, U, A, o, og, S, Au);
    TV rs = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (S.d[s] != TV(0)) rs += b[s] - Au[s];
    const int P = __ldg(T.oct_parent + og);
    B[cyc(P)] = scale * rs;
    U[cyc(P)] = S.ubar;
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_orestrict(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                    TV* __restrict__ B, TV scale) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    orestrict_octet<TV, TC, TW>(A, T, C, U, B, scale, o);
}

// Prolongation as its own launch (thread per child octet).
template <class TV, class TC>
__global__ void __launch_bounds__(OBLK) k_oprolong(LevelArgs A, Tables T, const TC* __restrict__ d,
                                                   TV* __restrict__ U) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    octet_prolong<TV>(d, U, c8 >> 3, U[cyc(__ldg(T.oct_parent + (c8 >> 3)))]);
}

// Outer vector: parent value = mean of the active children (composite operator, Sec. 3.1).
template <class TO, class TC>
__global__ void __launch_bounds__(OBLK) k_oavg(LevelArgs A, Tables T, const TC* __restrict__ d, TO* __restrict__ P) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    TO v[8], dd[8];
    ld8(P + c8, v);
    ldc8(d + c8, dd);
    TO s = TO(0);
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != TO(0)) { s += v[q]; ++n; }
    P[__ldg(T.oct_parent + (c8 >> 3))] = s * inv_count<TO>(n);
}

// The same child means for a vector kept as FP32 pairs (hi, lo): sum and division in pair
// arithmetic, the parent written as a normalised pair.
template <class TC>
__global__ void __launch_bounds__(OBLK) k_oavg_pp(LevelArgs A, Tables T, const TC* __restrict__ d,
                                                  float* __restrict__ hi, float* __restrict__ lo) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    float h[8], l[8], dd[8];
    ld8(hi + c8, h);
    ld8(lo + c8, l);
    ldc8(d + c8, dd);
    DF s{0.0f, 0.0f};
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != 0.0f) { df_acc(s, DF{h[q], l[q]}); ++n; }
    const DF m = df_norm(df_div_count(s, n));
    const int par = __ldg(T.oct_parent + (c8 >> 3));
    hi[par] = m.hi;
    lo[par] = m.lo;
}

// Composite leaf operator over all tree levels in one launch (block -> level lookup):
// Y = A p on leaves, 0 on inner cells; (p, A p) over leaves reduced into R.
struct OMultiLevel {
    int n;
    int off[MAXLEV];
    int noct[MAXLEV];
    int ni[MAXLEV];
    int boff[MAXLEV + 1];
};

// The grid is bounded (a few blocks per SM) and strides over the per-level octet blocks
// boff[], so the dot product reduces over at most gridDim partials.
template <class TO, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_oapply(OMultiLevel ML, Tables T, Coefs<TC, TW> C, const TO* __restrict__ P,
                                                 TO* __restrict__ Y, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    double dot = 0.0;
    const int nvb = ML.boff[ML.n];
    int l = 0;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    while (l + 1 < ML.n && vb >= ML.boff[l + 1]) ++l;
    const int o = (vb - ML.boff[l]) * OBLK + threadIdx.x;
    if (o < ML.noct[l]) {
        const int c8 = ML.off[l] + 8 * o;
        OctState<TO> S;
        load_octet<TO, TC, TW>(P, C, c8, S);
        octet_mean(S);
        TO Ap[8];
        const LevelArgs A{ML.off[l], 8 * ML.noct[l], ML.ni[l]};
        octet_Au<TO, TC, TW>(T, C, P, A, o, c8 >> 3, S, Ap);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const bool leaf = __ldg(T.child_oct + c8 + s) < 0;
            Y[c8 + s] = leaf ? Ap[s] : TO(0);
            if (leaf) dot += (double)S.u[s] * (double)Ap[s];
        }
    }
    }
    if (R.op != OP_NONE) red_finish(R, blockIdx.x, dot, 0.0, sh);
}

// ------------------------------------------------------------ conservative BF16 diagonal
// The diagonal of the BF16 coefficient set (kept in FP32): the FP64 remainder
// d - sum_f w_f over the faces that enter the sweep's stencil (the walls' weights; zero for
// an interior cell) minus the sum of the stored low-precision coefficients of those faces
// (BF16 faces, FP32 T-record weights).  A row of the stored operator then sums to the
// FP32-rounded remainder exactly, so BF16 storage keeps the constant null space of
// all-Neumann problems; rounding d and the faces independently would leave each row sum
// off by about 2^-9 d, which W-cycles amplify until PCG stalls.  Inactive cells keep 0.
template <class TL>
__global__ void __launch_bounds__(OBLK) k_diag_conservative(LevelArgs A, Tables T, Coefs<double, double> C64,
                                                            const TL* __restrict__ cxl, const TL* __restrict__ cyl,
                                                            const TL* __restrict__ czl, const float* __restrict__ twl,
                                                            float* __restrict__ dout) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o, og = c8 >> 3;
    double rem[8];
    float sl[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) { rem[s] = C64.d[c8 + s]; sl[s] = 0.0f; }
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    const double* c64[3] = {C64.cx, C64.cy, C64.cz};
    const TL* cl[3] = {cxl, cyl, czl};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), t = s | bit;
            const double c = c64[a][c8 + t];
            const float cf = tov(cl[a][c8 + t]);
            rem[s] += c; rem[t] += c;
            sl[s] += cf; sl[t] += cf;
        }
        const int v = nb[2 * a];
        if (v != -1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                rem[s] += c64[a][c8 + s];
                sl[s] += tov(cl[a][c8 + s]);
            }
        }
        const int w = nb[2 * a + 1];
        if (w >= 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit, n = A.off + 8 * w + clear_slot(a, q);
                rem[s] += c64[a][n];
                sl[s] += tov(cl[a][n]);
            }
        } else if (w <= -2) {
            const int t = T.trec[og];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit, idx = ((2 * a + 1) * 4 + q) * T.nt + t;
                rem[s] += C64.tw[idx];
                sl[s] += twl[idx];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) dout[c8 + s] = C64.d[c8 + s] == 0.0 ? 0.0f : (float)rem[s] - sl[s];
}

// ------------------------------------------------------------ outer apply, two lanes per octet
// The mixed-precision outer operator (FP64 vectors, FP32 coefficients) without the FP64
// pipe, which runs at 1/64 of the FP32 rate on this GPU: every binary64 value is split
// exactly into a pair of binary32 (hi, lo) with integer operations (48 significant bits
// kept), the stencil is evaluated in pair arithmetic with error-free transformations
// (TwoSum, TwoProd by FMA; T. J. Dekker, "A floating-point technique for extending the
// available precision", Numer. Math. 18, 1971), and only the final hi + lo of each output
// is one binary64 addition.  The flux form
//   (A u)_s = rem_s u_s + sum_f w_f (u_s - u_f)   (+ T ghosts (w_f/2)(ubar - u_K))
// computes every face difference before scaling it, so the rounding error is relative to
// the fluxes, not to d_s u_s.
// The remainder of a tree cell's diagonal after its stencil faces: rem = d + the sum of
// the stored FP32 coefficients (each -w_f) of the faces that enter the cell's stencil
// (internal faces, both neighbour faces, T sub-faces; a wall face enters only here),
// evaluated in FP64 from the FP64 diagonal and rounded once to FP32: 0 for an interior
// cell whose face weights are exact in FP32, the wall weight at a Dirichlet wall, a few
// ulps of w_f beside a rounded T-record weight, 0 for an inactive cell.  The flux form
// sum_f w_f (u_s - u_f) + rem u_s of the outer apply then carries the FP64 diagonal.
__global__ void __launch_bounds__(OBLK) k_remainder(LevelArgs A, Tables T, const double* __restrict__ d64,
                                                    Coefs<float, float> C, float* __restrict__ rem) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o, og = c8 >> 3;
    double r[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) r[s] = d64[c8 + s];
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    const float* cm[3] = {C.cx, C.cy, C.cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), t = s | bit;
            const double c = cm[a][c8 + t];
            r[s] += c;
            r[t] += c;
        }
        if (nb[2 * a] != -1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) r[clear_slot(a, q)] += (double)cm[a][c8 + clear_slot(a, q)];
        }
        const int w = nb[2 * a + 1];
        if (w >= 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) r[clear_slot(a, q) | bit] += (double)cm[a][A.off + 8 * w + clear_slot(a, q)];
        } else if (w <= -2) {
            const int t = T.trec[og];
#pragma unroll
            for (int q = 0; q < 4; ++q) r[clear_slot(a, q) | bit] += (double)C.tw[((2 * a + 1) * 4 + q) * T.nt + t];
        }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) rem[c8 + s] = (float)r[s];
}

constexpr int OBLK2 = 128;   // threads per block of the two-lane apply: 64 octets

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float f4at(const float4& v, int q) {
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}
__device__ __forceinline__ DF shfl_df(unsigned m, DF v) {
    return DF{__shfl_xor_sync(m, v.hi, 1), __shfl_xor_sync(m, v.lo, 1)};
}

// Vectors of the outer apply.  VecD: binary64 values, split into pairs on load (48 bits
// kept).  VecP: the pair itself in two FP32 arrays hi, lo (value hi + lo, exact in
// binary64), the form in which the mixed PCG keeps its search direction p, so that the
// apply does not split.  OutD: results rounded back to binary64.
struct VecD {
    const double* __restrict__ p;
    __device__ __forceinline__ DF one(int i) const { return df_split(p[i]); }
    __device__ __forceinline__ void two(int i, DF& a, DF& b) const {
        const double2 v = *reinterpret_cast<const double2*>(p + i);
        a = df_split(v.x);
        b = df_split(v.y);
    }
    __device__ __forceinline__ void four(int i, DF (&v)[4]) const {
        two(i, v[0], v[1]);
        two(i + 2, v[2], v[3]);
    }
};
struct VecP {
    const float* __restrict__ hi;
    const float* __restrict__ lo;
    __device__ __forceinline__ DF one(int i) const { return DF{hi[i], lo[i]}; }
    __device__ __forceinline__ void two(int i, DF& a, DF& b) const {
        const float2 h = *reinterpret_cast<const float2*>(hi + i), l = *reinterpret_cast<const float2*>(lo + i);
        a = DF{h.x, l.x};
        b = DF{h.y, l.y};
    }
    __device__ __forceinline__ void four(int i, DF (&v)[4]) const {
        const float4 h = *reinterpret_cast<const float4*>(hi + i), l = *reinterpret_cast<const float4*>(lo + i);
        v[0] = DF{h.x, l.x}; v[1] = DF{h.y, l.y}; v[2] = DF{h.z, l.z}; v[3] = DF{h.w, l.w};
    }
};
struct OutD {
    double* __restrict__ y;
    __device__ __forceinline__ void zero4(int i) const {
        reinterpret_cast<double4*>(y + i)[0] = make_double4(0.0, 0.0, 0.0, 0.0);
    }
    // a normalised pair per cell, 0 where keep is false
    __device__ __forceinline__ void put4(int i, const DF (&v)[4], int keep) const {
        double w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = ((keep >> q) & 1) ? df_to_double(v[q]) : 0.0;
        reinterpret_cast<double4*>(y + i)[0] = make_double4(w[0], w[1], w[2], w[3]);
    }
};
// One z layer (4 cells, slots 4z..4z+3) of the pair-of-FP32 outer apply: the two lanes
// of a pair (mask pm) hold the two layers of one octet and trade their values for the
// faces between the layers.  Per face: the exact difference of the two values by TwoSum,
// its product with the FP32 coefficient by FMA, pair accumulation; the diagonal enters as
// the remainder from k_remainder, the leaf flags come from the 1-byte cell flags.
template <class V, class O>
__device__ __forceinline__ void layer_apply_df(const Tables& T, const Coefs<float, float>& C,
                                               const float* __restrict__ rem, const uint8_t* __restrict__ flags,
                                               const V& P, const O& Y, int off, int ni, int o, int z, unsigned pm,
                                               DF& dot, DF& sum) {
    const int c8 = off + 8 * o, og = c8 >> 3, cz0 = c8 + 4 * z;
    const uint32_t fl = __ldg(reinterpret_cast<const uint32_t*>(flags + cz0));
    const int leafm = (int)((fl & 1u) | ((fl >> 7) & 2u) | ((fl >> 14) & 4u) | ((fl >> 21) & 8u));
    const int leafo = __shfl_xor_sync(pm, leafm, 1);
    if ((leafm | leafo) == 0) {
        // no leaf in the octet: the composite operator has no row here
        Y.zero4(cz0);
        return;
    }
    int nb[6];
    octet_neighbours(T, ni, o, og, nb);
    DF u[4], uo[4], acc[4];
    P.four(cz0, u);
#pragma unroll
    for (int q = 0; q < 4; ++q) { uo[q] = shfl_df(pm, u[q]); acc[q] = DF{0.0f, 0.0f}; }
    const float4 cx = ldg4(C.cx + cz0), cy = ldg4(C.cy + cz0), czv = ldg4(C.cz + cz0);
    const float4 rm = ldg4(rem + cz0);
    // the mean of the octet's active cells, for T ghosts (pair-uniform: both lanes share nb)
    DF ubar{0.0f, 0.0f};
    if (nb[0] <= -2 || nb[1] <= -2 || nb[2] <= -2 || nb[3] <= -2 || nb[4] <= -2 || nb[5] <= -2) {
        const float4 d = ldg4(C.d + cz0);
        DF sm{0.0f, 0.0f};
        int n = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (f4at(d, q) != 0.0f) { df_acc(sm, u[q]); ++n; }
        df_acc(sm, shfl_df(pm, sm));
        n += __shfl_xor_sync(pm, n, 1);
        ubar = df_div_count(sm, n);
    }
    // faces inside the layer: x between q and q|1, y between q and q|2 (coefficient kept
    // by the + cell)
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
        const DF f = df_scale(df_diff(u[q], u[q + 1]), -f4at(cx, q + 1));
        df_acc(acc[q], f);
        df_acc(acc[q + 1], DF{-f.hi, -f.lo});
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const DF f = df_scale(df_diff(u[q], u[q + 2]), -f4at(cy, q + 2));
        df_acc(acc[q], f);
        df_acc(acc[q + 2], DF{-f.hi, -f.lo});
    }
    // faces between the layers: the coefficient is the upper layer's c_z-
    {
        float czu[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float mine = f4at(czv, q), other = __shfl_xor_sync(pm, mine, 1);
            czu[q] = z ? mine : other;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) df_acc(acc[q], df_scale(df_diff(u[q], uo[q]), -czu[q]));
    }
    // x and y faces of the octet: the - face meets the neighbour's + side, whose cells are
    // those with the bit set; the + face meets the neighbour's - side, which keeps the
    // coefficients
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int bit = 1 << a;
        const float4& cown = a == 0 ? cx : cy;
        const float* cg = a == 0 ? C.cx : C.cy;
        const int v = nb[2 * a];
        if (v >= 0) {
            const int pn = off + 8 * v + 4 * z;
            DF nv[2];
            if (a == 0) { nv[0] = P.one(pn + 1); nv[1] = P.one(pn + 3); }
            else P.two(pn + 2, nv[0], nv[1]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = a == 0 ? 2 * k : k;            // cells with the bit clear
                df_acc(acc[q], df_scale(df_diff(u[q], nv[k]), -f4at(cown, q)));
            }
        } else if (v <= -2) {
            const DF gk = df_diff(P.one(-2 - v), ubar);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = a == 0 ? 2 * k : k;
                df_acc(acc[q], df_scale(gk, 0.5f * f4at(cown, q)));
            }
        }
        const int w = nb[2 * a + 1];
        if (w >= 0) {
            const int n8 = off + 8 * w + 4 * z;
            DF nv[2];
            if (a == 0) { nv[0] = P.one(n8); nv[1] = P.one(n8 + 2); }
            else P.two(n8, nv[0], nv[1]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = a == 0 ? 2 * k + 1 : k + 2;    // cells with the bit set
                const int qn = q & ~bit;
                df_acc(acc[q], df_scale(df_diff(u[q], nv[k]), -__ldg(cg + n8 + qn)));
            }
        } else if (w <= -2) {
            const DF gk = df_diff(P.one(-2 - w), ubar);
            const int t = __ldg(T.trec + og);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = a == 0 ? 2 * k + 1 : k + 2;
                const int sub = sub_index(a, 4 * z + q);
                df_acc(acc[q], df_scale(gk, 0.5f * __ldg(C.tw + ((2 * a + 1) * 4 + sub) * T.nt + t)));
            }
        }
    }
    // z face of this layer: the - face for the lower layer (the neighbour's upper layer,
    // own coefficients), the + face for the upper one (the neighbour's lower layer and its
    // coefficients)
    {
        const int v = z ? nb[5] : nb[4];
        if (v >= 0) {
            const int n8 = off + 8 * v;
            DF nv[4];
            P.four(n8 + 4 * (1 - z), nv);
            const float4 cc = z ? ldg4(C.cz + n8) : czv;
            df_acc(acc[0], df_scale(df_diff(u[0], nv[0]), -cc.x));
            df_acc(acc[1], df_scale(df_diff(u[1], nv[1]), -cc.y));
            df_acc(acc[2], df_scale(df_diff(u[2], nv[2]), -cc.z));
            df_acc(acc[3], df_scale(df_diff(u[3], nv[3]), -cc.w));
        } else if (v <= -2) {
            const DF gk = df_diff(P.one(-2 - v), ubar);
            const int t = z ? __ldg(T.trec + og) : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float c = z ? __ldg(C.tw + (5 * 4 + q) * T.nt + t) : f4at(czv, q);
                df_acc(acc[q], df_scale(gk, 0.5f * c));
            }
        }
    }
    DF out[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool leaf = (leafm >> q) & 1;
        DF au = acc[q];
        df_acc(au, df_scale(u[q], f4at(rm, q)));
        out[q] = df_norm(au);
        if (leaf) {
            df_acc(dot, df_mul(u[q], out[q]));
            df_acc(sum, out[q]);
        }
    }
    Y.put4(cz0, out, leafm);
}

// Y = A P over all tree levels (FP64 vectors, FP32 coefficients), two lanes per octet;
// (P, A P) and the sum of A P over the leaves reduced into R.  Blocks of OBLK2 threads take the octet blocks
// (64 octets) of OMultiLevel and stride over them.
template <class V, class O>
__global__ void __launch_bounds__(OBLK2, 8) k_oapply_df2(OMultiLevel ML, Tables T, Coefs<float, float> C,
                                                         const float* __restrict__ rem,
                                                         const uint8_t* __restrict__ flags, V P, O Y, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    DF dot{0.0f, 0.0f}, sum{0.0f, 0.0f};
    const int nvb = ML.boff[ML.n];
    const int z = threadIdx.x & 1;
    const unsigned pm = 3u << (threadIdx.x & 30);
    int l = 0;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        while (l + 1 < ML.n && vb >= ML.boff[l + 1]) ++l;
        const int o = (vb - ML.boff[l]) * OBLK + (threadIdx.x >> 1);
        if (o < ML.noct[l]) layer_apply_df(T, C, rem, flags, P, Y, ML.off[l], ML.ni[l], o, z, pm, dot, sum);
    }
    if (R.op != OP_NONE) red_finish(R, blockIdx.x, df_to_double(dot), df_to_double(sum), sh);
}

// ------------------------------------------------------------ transposed operator
// A^T x = A x + (A^T - A) x, the correction summed over the T sub-faces f (fine leaf i,
// coarser leaf K, P = parent of i, c_f = w_f / 2):
//   c_f (x_i - x_K) a_P  -  c_f (xbar_P - x_K) (e_i - e_K),
// xbar_P = a_P^T x the mean of P's children (written into x's inner cells by the
// averaging pass of the forward apply).  Three gathers, each output written by one thread:
//   k_tfine:   per T octet: y_i -= sum c_f (xbar_P - x_K); tseed[P] = sum c_f (x_i - x_K);
//   k_tcoarse: per coarse leaf K: y_K += sum c_f ((xbar_P - x_K) - (x_i - x_K));
//   k_tdesc:   per octet below a T parent: every leaf gets sum over its ancestors A of
//              tseed[A] 8^-(depth difference)  (tseed is zero away from the T parents).
// c_f comes from the same coefficients as the forward operator (the fine cell's c_{a-} for a
// face on the octet's - side, the T record for the + side), so the result is the exact
// transpose of the operator k_oapply applies.
template <class TO, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_tfine(Tables T, Coefs<TC, TW> C, const int32_t* __restrict__ t_oct,
                                                 TO* __restrict__ X, TO* __restrict__ Y, double* __restrict__ tseed) {
    pdl_enter();
    const int q = blockIdx.x * OBLK + threadIdx.x;
    if (q >= T.nt) return;
    const int og = __ldg(t_oct + q);
    const int c8 = 8 * og;
    const int P = __ldg(T.oct_parent + og);
    const double xbar = (double)X[P];
    double yi[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double tacc = 0.0;
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int v = __ldg(T.nbr + dir * T.noct + og);
        if (v > -2) continue;
        const double xK = (double)X[-2 - v];
        const int a = dir >> 1, bit = 1 << a;
        const TC* cm = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int s = clear_slot(a, qq) | ((dir & 1) ? bit : 0);
            const double cf = (dir & 1) ? (double)tov(__ldg(C.tw + ((2 * a + 1) * 4 + qq) * T.nt + q))
                                        : (double)tov(__ldg(cm + c8 + s));
            const double c = -0.5 * cf;
            tacc += c * ((double)X[c8 + s] - xK);
            yi[s] -= c * (xbar - xK);
        }
    }
    tseed[P] = tacc;
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (yi[s] != 0.0) Y[c8 + s] = TO((double)Y[c8 + s] + yi[s]);
}

template <class TO, class TC, class TW>
__global__ void k_tcoarse(Tables T, Coefs<TC, TW> C, OMultiLevel ML, const int8_t* __restrict__ level,
                          const int32_t* __restrict__ tcoarse, int n, const TO* __restrict__ X, TO* __restrict__ Y) {
    pdl_enter();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int K = __ldg(tcoarse + q);
    const int m = level[K];
    const int off = ML.off[m], sK = K & 7, og = K >> 3, o = (K - off) >> 3;
    int nb[6];
    octet_neighbours(T, ML.ni[m], o, og, nb);
    const double xK = (double)X[K];
    double acc = 0.0;
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int a = dir >> 1, bit = 1 << a;
        const bool plus = dir & 1;
        int Q = -1;
        if (((sK & bit) != 0) != plus) Q = plus ? K + bit : K - bit;
        else if (nb[dir] >= 0) Q = off + 8 * nb[dir] + (sK ^ bit);
        if (Q < 0) continue;
        const int co = __ldg(T.child_oct + Q);
        if (co < 0) continue;
        const double xbar = (double)X[Q];
        const TC* cm = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
        const int t = plus ? 0 : __ldg(T.trec + co);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int s = clear_slot(a, qq) | (plus ? 0 : bit);
            const int i = 8 * co + s;
            const double cf = plus ? (double)tov(__ldg(cm + i))
                                   : (double)tov(__ldg(C.tw + ((2 * a + 1) * 4 + qq) * T.nt + t));
            acc += -0.5 * cf * ((xbar - xK) - ((double)X[i] - xK));
        }
    }
    Y[K] = TO((double)Y[K] + acc);
}

template <class TO>
__global__ void k_tdesc(Tables T, const int32_t* __restrict__ tdesc, int n, int ntree,
                        const uint8_t* __restrict__ flags, const double* __restrict__ tseed, TO* __restrict__ Y) {
    pdl_enter();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int og = __ldg(tdesc + q);
    double acc = 0.0, w = 0.125;
    int A = __ldg(T.oct_parent + og);
    while (A >= 0 && A < ntree) {
        acc += tseed[A] * w;
        w *= 0.125;
        A = __ldg(T.oct_parent + (A >> 3));
    }
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (flags[8 * og + s] & 1) Y[8 * og + s] = TO((double)Y[8 * og + s] + acc);
}

// ------------------------------------------------------------ transposed cycle
// M^T, the transpose of the mu-cycle (a linear map r -> z from zero), for preconditioning
// the adjoint system: A^T M^T = (M A)^T has the spectrum of A M.  The transposed steps of
// Alg. 4 run in reverse order on adjoint states (ubar in U, bbar in B).  The level operator
// A^m of a fine cell s with T faces (coarser leaf K, octet mean ubar over n active cells)
// has the row  (d_s + W_s) u_s + c_f/2 u_K - W_s/(2n) sum_active u_j + regular faces,
// W_s = sum of s's T-face coefficients; so
//   (A^m^T X)_j = (d_j + W_j) X_j + sum_regular c X_nb - [j active] sum_s W_s X_s / (2n)
// within the level, and the coarser leaf K receives sum (c_f/2) X_s (B^m^T X).

// Y = A^m^T X for the 8 cells of octet o (see above); X is read, Y returned.
template <class TV, class TC, class TW>
__device__ __forceinline__ void octet_AT(const Tables& T, const Coefs<TC, TW>& C, const TV* X, const LevelArgs& A,
                                         int o, int og, TV (&Y)[8]) {
    const int c8 = A.off + 8 * o;
    TV x[8], d[8], cm[3][8], W[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = X[c8 + q];
    ldc8(C.d + c8, d);
    ldc8(C.cx + c8, cm[0]);
    ldc8(C.cy + c8, cm[1]);
    ldc8(C.cz + c8, cm[2]);
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    int nact = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) { W[s] = TV(0); nact += d[s] != TV(0) ? 1 : 0; }
    int t = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        if (nb[2 * a] <= -2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) W[clear_slot(a, q)] += cm[a][clear_slot(a, q)];
        }
        if (nb[2 * a + 1] <= -2) {
            if (t < 0) t = __ldg(T.trec + og);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                W[clear_slot(a, q) | bit] += TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + q) * T.nt + t)));
        }
    }
    TV tO = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s) { Y[s] = (d[s] + W[s]) * x[s]; tO += W[s] * x[s]; }
    tO = tO * TV(0.5) * inv_count<TV>(nact);
    const int off = A.off;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), u = s | bit;
            const TV c = cm[a][u];
            Y[s] += c * x[u];
            Y[u] += c * x[s];
        }
        const int v = nb[2 * a];
        if (v >= 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Y[s] += cm[a][s] * X[off + 8 * v + (s | bit)];
            }
        }
        const int w = nb[2 * a + 1];
        if (w >= 0) {
            const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Y[s | bit] += TV(tov(__ldg(cc + off + 8 * w + s))) * X[off + 8 * w + s];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (d[s] != TV(0)) Y[s] -= tO;
}

// T faces of an octet in the transposed kernels: W[s] += the coefficients of cell s's T
// faces, and (acc) the coarser leaf K's share B^m^T v, the sum of (c_f / 2) v_s over the 4
// cells of the face, added to the octet's slot Tacc[dir][record] (collected by kt_tgather).
// Returns the octet's T record (-1 without T faces).
template <class TV, class TC, class TW>
__device__ __forceinline__ int t_faces(const Tables& T, const Coefs<TC, TW>& C, const TV (&cm)[3][8], const TV (&v)[8],
                                       const int (&nb)[6], int og, TV (&W)[8], TV* __restrict__ Tacc, int acc) {
    bool any = false;
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) any |= nb[dir] <= -2;
    if (!any) return -1;
    const int t = __ldg(T.trec + og);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        if (nb[2 * a] <= -2) {
            TV f = TV(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                W[s] += cm[a][s];
                f += cm[a][s] * v[s];
            }
            if (acc) Tacc[(2 * a) * T.nt + t] += TV(0.5) * f;
        }
        if (nb[2 * a + 1] <= -2) {
            TV f = TV(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit;
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + q) * T.nt + t)));
                W[s] += cf;
                f += cf * v[s];
            }
            if (acc) Tacc[(2 * a + 1) * T.nt + t] += TV(0.5) * f;
        }
    }
    return t;
}

// Transposed colour sweep in one launch, reading ubar from Uin and writing Uout (ping-pong,
// so that V = Uin / d on the colour's active cells of a neighbouring octet can be recomputed
// here instead of being stored): bbar += V, Uout = Uin - A^m^T V.  Only cells of the other
// colour see V across a face (red-black), so only their neighbour values are fetched.
template <class TV>
__device__ __forceinline__ TV colour_v(TV u, TV d, bool on) {
    return (on && d != TV(0)) ? u / d : TV(0);
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) kt_fsweep(LevelArgs A, Tables T, Coefs<TC, TW> C, const TV* __restrict__ Uin,
                                                  TV* __restrict__ Uout, TV* __restrict__ B, TV* __restrict__ Tacc,
                                                  int colour, int acc) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o, og = c8 >> 3;
    TV u[8], d[8], cm[3][8], v[8], W[8], Y[8];
    ld8(Uin + c8, u);
    ldc8(C.d + c8, d);
    ldc8(C.cx + c8, cm[0]);
    ldc8(C.cy + c8, cm[1]);
    ldc8(C.cz + c8, cm[2]);
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    int nact = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        nact += d[s] != TV(0) ? 1 : 0;
        v[s] = colour_v(u[s], d[s], (__popc(s) & 1) == colour);
        W[s] = TV(0);
    }
    t_faces(T, C, cm, v, nb, og, W, Tacc, acc);
    TV tO = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s) { Y[s] = (d[s] + W[s]) * v[s]; tO += W[s] * v[s]; }
    tO = tO * TV(0.5) * inv_count<TV>(nact);
    const int off = A.off;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), w = s | bit;
            const TV c = cm[a][w];
            Y[s] += c * v[w];
            Y[w] += c * v[s];
        }
        // neighbouring octets' faces read as layers (ld_layer: a z layer in one vector
        // load, a y layer in two), both colours fetched, the colour's cells used
        const int vn = nb[2 * a];
        if (vn >= 0) {
            const int n8 = off + 8 * vn;
            TV nu[4];
            typename DiagOf<TC>::type ndr[4];
            ld_layer(Uin + n8, a, 1, true, nu);
            ld_layer(C.d + n8, a, 1, true, ndr);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q), ns = s | bit;
                if ((__popc(ns) & 1) != colour) continue;   // neighbour cell not of the colour
                Y[s] += cm[a][s] * colour_v(nu[q], TV(tov(ndr[q])), true);
            }
        }
        const int wn = nb[2 * a + 1];
        if (wn >= 0) {
            const int n8 = off + 8 * wn;
            const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
            TV nu[4];
            typename DiagOf<TC>::type ndr[4];
            TC ncr[4];
            ld_layer(Uin + n8, a, 0, true, nu);
            ld_layer(C.d + n8, a, 0, true, ndr);
            ld_layer(cc + n8, a, 0, true, ncr);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                if ((__popc(s) & 1) != colour) continue;
                Y[s | bit] += TV(tov(ncr[q])) * colour_v(nu[q], TV(tov(ndr[q])), true);
            }
        }
    }
    TV b[8];
    ld8(B + c8, b);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        Y[s] = u[s] - Y[s] + (d[s] != TV(0) ? tO : TV(0));
        b[s] += v[s];
    }
    st8(Uout + c8, Y);
    st8(B + c8, b);
}

// transposed colour sweep, part 1: V = ubar / d on the active cells of the colour (0
// elsewhere), bbar += V
template <class TV, class TC, class TW>
__device__ __forceinline__ void sweep_v_octet(const LevelArgs& A, const Coefs<TC, TW>& C, const TV* U, TV* B, TV* V,
                                              int colour, int o) {
    const int c8 = A.off + 8 * o;
    TV u[8], b[8], d[8], v[8];
    ld8(U + c8, u);
    ld8(B + c8, b);
    ldc8(C.d + c8, d);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        v[s] = ((__popc(s) & 1) == colour && d[s] != TV(0)) ? u[s] / d[s] : TV(0);
        b[s] += v[s];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) V[c8 + q] = v[q];
    st8(B + c8, b);
}

// ubar_K -= the slots Tacc of the fine T octets beside K, for the coarser leaves K listed in
// tcoarse[k0, k1) (those of one level; the fine octets are one level finer); the slots
// are zeroed (each belongs to one K).
template <class TV>
__global__ void kt_tgather(Tables T, OMultiLevel ML, const int8_t* __restrict__ level,
                           const int32_t* __restrict__ tcoarse, int k0, int k1, TV* __restrict__ U,
                           TV* __restrict__ Tacc) {
    pdl_enter();
    const int q = k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k1) return;
    const int K = __ldg(tcoarse + q);
    const int m = level[K];
    const int off = ML.off[m], sK = K & 7, og = K >> 3, o = (K - off) >> 3;
    int nb[6];
    octet_neighbours(T, ML.ni[m], o, og, nb);
    TV acc = TV(0);
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int a = dir >> 1, bit = 1 << a;
        const bool plus = dir & 1;
        int Q = -1;
        if (((sK & bit) != 0) != plus) Q = plus ? K + bit : K - bit;
        else if (nb[dir] >= 0) Q = off + 8 * nb[dir] + (sK ^ bit);
        if (Q < 0) continue;
        const int co = __ldg(T.child_oct + Q);
        if (co < 0) continue;
        // K lies on the - side of the fine octet when Q is on K's + side
        const int slot = (plus ? 2 * a : 2 * a + 1) * T.nt + __ldg(T.trec + co);
        acc += Tacc[slot];
        Tacc[slot] = TV(0);
    }
    U[K] -= acc;
}

// transposed prolongation (u^m += P (u^{m-1} - u*) on active children) and correction:
// per octet of level m with parent P: corr = sum of ubar over its active cells;
// ubar_P += corr; UST_P = -corr (the adjoint of u*, completed after the recursion)
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) kt_prolong(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                   TV* __restrict__ UST) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    TV u[8], d[8];
    ld8(U + c8, u);
    ldc8(C.d + c8, d);
    TV corr = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (d[s] != TV(0)) corr += u[s];
    const int P = __ldg(T.oct_parent + (c8 >> 3));
    U[P] += corr;
    UST[P] = -corr;
}

// transposed FAS restriction, part 1, over the cells of level m-1: for a cell with
// children, g = bbar (then 0), UST += ubar (then 0: u^{m-1} was overwritten by u*);
// G = g there and 0 on leaves
template <class TV>
__global__ void kt_restrict_g(LevelArgs A, Tables T, TV* __restrict__ U, TV* __restrict__ B, TV* __restrict__ UST,
                              TV* G) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.ncell) return;
    const int c = A.off + i;
    if (__ldg(T.child_oct + c) >= 0) {
        G[c] = B[c];
        B[c] = TV(0);
        UST[c] += U[c];
        U[c] = TV(0);
    } else {
        G[c] = TV(0);
    }
}

// transposed FAS restriction, part 2, over the cells of level m-1: v = A^{m-1}^T G (the
// rows with children are regular, so no T terms arise); UST += v on cells with children,
// ubar += v on the others
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) kt_restrict_v(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                      TV* __restrict__ UST, const TV* G) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    TV y[8];
    octet_AT<TV, TC, TW>(T, C, G, A, o, c8 >> 3, y);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        if (__ldg(T.child_oct + c8 + s) >= 0) UST[c8 + s] += y[s];
        else U[c8 + s] += y[s];
    }
}

// transposed FAS restriction, part 3, per octet of level m with parent P: on the active
// cells rbar = (beta/alpha) G_P, bbar += rbar, ubar += UST_P / n (transpose of u* = the
// mean of the active children), then ubar -= A^m^T rbar (the residual's transpose), with
// rbar of a neighbouring cell recomputed from its parent's G (G held in X on level m-1).
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) kt_restrict_c(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                      TV* __restrict__ B, const TV* __restrict__ UST,
                                                      const TV* __restrict__ G, TV* __restrict__ Tacc, TV scale,
                                                      int acc) {
    pdl_enter();
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o, og = c8 >> 3;
    const int P = __ldg(T.oct_parent + og);
    TV d[8], cm[3][8], v[8], W[8], Y[8];
    ldc8(C.d + c8, d);
    ldc8(C.cx + c8, cm[0]);
    ldc8(C.cy + c8, cm[1]);
    ldc8(C.cz + c8, cm[2]);
    int nb[6];
    octet_neighbours(T, A.ni, o, og, nb);
    int nact = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) nact += d[s] != TV(0) ? 1 : 0;
    const TV r = scale * G[P], us = UST[P] * inv_count<TV>(nact);
#pragma unroll
    for (int s = 0; s < 8; ++s) { v[s] = d[s] != TV(0) ? r : TV(0); W[s] = TV(0); }
    t_faces(T, C, cm, v, nb, og, W, Tacc, acc);
    TV tO = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s) { Y[s] = (d[s] + W[s]) * v[s]; tO += W[s] * v[s]; }
    tO = tO * TV(0.5) * inv_count<TV>(nact);
    const int off = A.off;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), w = s | bit;
            const TV c = cm[a][w];
            Y[s] += c * v[w];
            Y[w] += c * v[s];
        }
        const int vn = nb[2 * a];
        if (vn >= 0) {
            const int n8 = off + 8 * vn;
            const TV rn = scale * G[__ldg(T.oct_parent + (n8 >> 3))];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q), ns = s | bit;
                if (TV(tov(__ldg(C.d + n8 + ns))) != TV(0)) Y[s] += cm[a][s] * rn;
            }
        }
        const int wn = nb[2 * a + 1];
        if (wn >= 0) {
            const int n8 = off + 8 * wn;
            const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
            const TV rn = scale * G[__ldg(T.oct_parent + (n8 >> 3))];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                if (TV(tov(__ldg(C.d + n8 + s))) != TV(0)) Y[s | bit] += TV(tov(__ldg(cc + n8 + s))) * rn;
            }
        }
    }
    TV u[8], b[8];
    ld8(U + c8, u);
    ld8(B + c8, b);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const bool act = d[s] != TV(0);
        b[s] += v[s];
        u[s] += (act ? us + tO : TV(0)) - Y[s];
    }
    st8(U + c8, u);
    st8(B + c8, b);
}

// transposed smoothing of the coarsest level in one CTA: 2 nsweep colour sweeps, the first
// 2 n_a of them in the colour order 0, 1, the rest 1, 0 (the reverse of the forward
// coarsest smoothing); the level has no coarser leaves
template <class TV, class TC, class TW>
__global__ void kt_coarsest(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* U, TV* B, TV* V, int n_a, int nsweep) {
    pdl_enter();
    const int noct = A.ncell / 8;
    for (int k = 0; k < 2 * nsweep; ++k) {
        const int colour = k < 2 * n_a ? (k & 1) : 1 - (k & 1);
        for (int o = threadIdx.x; o < noct; o += blockDim.x) sweep_v_octet<TV, TC, TW>(A, C, U, B, V, colour, o);
        __syncthreads();
        for (int o = threadIdx.x; o < noct; o += blockDim.x) {
            const int c8 = A.off + 8 * o;
            TV y[8];
            octet_AT<TV, TC, TW>(T, C, V, A, o, c8 >> 3, y);
#pragma unroll
            for (int q = 0; q < 8; ++q) U[c8 + q] -= y[q];
        }
        __syncthreads();
    }
}

// M^T input: U = the leaf values of Z (0 on inner cells), B = 0, over the tree cells
template <class TV, class TZ>
__global__ void kt_seed(int n, const uint8_t* __restrict__ flags, const TZ* Z, TV* __restrict__ U, TV* B) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TV z = TV(Z[i]);   // Z may be B itself
    U[i] = (flags[i] & 1) ? z : TV(0);
    B[i] = TV(0);
}

// Coarsest level (Alg. 4, l = 0): one CTA, one thread per octet, nu sweeps (half
// red->black, half black->red), each a pass separated by __syncthreads; fas completes
// the FAS right-hand side first; prolong prolongs onto the finer level at the end.
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(256) k_ocoarsest(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                    TV* __restrict__ B, int nu, int fas, int prolong) {
    pdl_enter();
    const int noct = A.ncell / 8;
    auto pass = [&](int colour, bool fixb) {
        for (int o = threadIdx.x; o < noct; o += blockDim.x) {
            const int c8 = A.off + 8 * o;
            OctState<TV> S;
            load_octet<TV, TC, TW, true>(U, C, c8, S);
            octet_mean(S);
            TV b[8], Au[8];
            ldv8<true>(B, c8, b);
            octet_Au<TV, TC, TW, true>(T, C, U, A, o, c8 >> 3, S, Au);
            if (fixb) {
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    if (T.child_oct[c8 + s] >= 0) B[cyc(c8 + s)] = b[s] + Au[s];
            } else {
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    if (((__popc(s) & 1) == colour) && S.d[s] != TV(0))
                        U[cyc(c8 + s)] = S.u[s] + divide(b[s] - Au[s], S.d[s]);
            }
        }
        __syncthreads();
    };
    if (fas) pass(0, true);
    const int half = nu / 2;
    for (int it = 0; it < half; ++it) { pass(0, false); pass(1, false); }
    for (int it = half; it < nu; ++it) { pass(1, false); pass(0, false); }
    if (prolong) {
        for (int c = threadIdx.x; c < A.ncell; c += blockDim.x) {
            const int co = T.child_oct[A.off + c];
            if (co >= 0) octet_prolong<TV>(C.d, U, co, U[cyc(A.off + c)]);
        }
    }
}

// ------------------------------------------------------------------ coarse tail
// The smallest uniform levels (m < 0) run their whole sub-cycle of Alg. 4 in one CTA with
// u, b and the coefficients in shared memory, one thread per octet.  On these levels the
// octets are lexicographic, so neighbours, parents and children are arithmetic and no
// table is read.  Shared arrays are slot-major (index sbase + s * noct + o) so that the
// threads of a warp, which own consecutive octets, touch consecutive banks.
struct TailLevel {
    int off;      // first global cell
    int ni;       // octets per axis
    int sbase;    // first element in the shared arrays
};

struct TailArgs {
    int nlev;                 // L[0] = top (finest) tail level ... L[nlev-1] = coarsest
    TailLevel L[MAXLEV];
    int ncell;
    const int* sched;         // passes of the sub-cycle: 8 * level index + pass kind
    int nsched;
    int fas, prolong;
    int up_off, up_ni;        // the uniform level above the tail (prolongation target)
};

constexpr int TAIL_SCHED_SH = 256;   // schedules up to this length are kept in shared memory

template <class TV>
struct TailMem {
    TV *u, *b, *d, *cm[3];
};

__device__ __forceinline__ int tail_noct(const TailLevel& L) { return L.ni * L.ni * L.ni; }

template <class TV>
__device__ __forceinline__ void tail_octet_Au(const TailMem<TV>& M, const TailLevel& L, int o, const TV (&u)[8],
                                              const TV (&d)[8], const TV (&cm)[3][8], TV (&Au)[8]) {
    const int ni = L.ni, no = ni * ni * ni;
    int I, J, K;
    octet_coords(o, ni, I, J, K);
    const int crd[3] = {I, J, K};
    const int stride[3] = {1, ni, ni * ni};
#pragma unroll
    for (int s = 0; s < 8; ++s) Au[s] = d[s] * u[s];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = clear_slot(a, q), t = s | bit;
            Au[s] += cm[a][t] * u[t];
            Au[t] += cm[a][t] * u[s];
        }
        if (crd[a] > 0) {
            const int nbo = L.sbase + o - stride[a];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += cm[a][s] * M.u[nbo + (s | bit) * no];
            }
        }
        if (crd[a] < ni - 1) {
            const int nbo = L.sbase + o + stride[a];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s | bit] += M.cm[a][nbo + s * no] * M.u[nbo + s * no];
            }
        }
    }
}

// parent (shared index) of octet o of level L, on the coarser tail level P
__device__ __forceinline__ int tail_parent(const TailLevel& L, const TailLevel& P, int o) {
    int I, J, K;
    octet_coords(o, L.ni, I, J, K);
    const int po = (I >> 1) + P.ni * ((J >> 1) + P.ni * (K >> 1));
    const int slot = (I & 1) | ((J & 1) << 1) | ((K & 1) << 2);
    return P.sbase + slot * tail_noct(P) + po;
}

enum { TP_SWEEP0 = 0, TP_SWEEP1 = 1, TP_FIXB = 2, TP_RESTRICT = 3, TP_PROLONG = 4 };

// Colour sweep of a tail level over the colour's cells only: work item i is the k-th slot of
// the colour (s = 2k + (parity(k) xor colour): 0, 3, 5, 6 or 1, 2, 4, 7) of octet o, so
// the threads do no work on the other colour (one thread per octet would evaluate all 8
// stencils).  The sum runs in the octet form's order (per axis: octet partner, then the
// neighbouring octet).  Shared index of cell (o, s) is sbase + s * no + o.
template <class TV>
__device__ __forceinline__ void tail_sweep_cell(const TailMem<TV>& M, const TailLevel& L, int colour, int i) {
    const int ni = L.ni, no = ni * ni * ni;
    const bool p2 = (no & (no - 1)) == 0;
    const int sh = p2 ? __ffs(no) - 1 : 0;
    const int k = p2 ? (i >> sh) : i / no;
    const int o = i - k * no;
    const int s = 2 * k + ((__popc(k) & 1) ^ colour);
    const int q = L.sbase + s * no + o;
    const TV dd = M.d[q];
    if (dd == TV(0)) return;
    int crd[3];
    octet_coords(o, ni, crd[0], crd[1], crd[2]);
    const int stride[3] = {1, ni, ni * ni};
    TV Au = dd * M.u[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const int t = s ^ bit;
        const int qi = L.sbase + t * no + o;                // partner in the octet
        if (s & bit) {
            Au += M.cm[a][q] * M.u[qi];
            if (crd[a] < ni - 1) {
                const int qo = qi + stride[a];               // slot t of the + octet
                Au += M.cm[a][qo] * M.u[qo];
            }
        } else {
            Au += M.cm[a][qi] * M.u[qi];
            if (crd[a] > 0) Au += M.cm[a][q] * M.u[qi - stride[a]];   // slot t of the - octet
        }
    }
    M.u[q] = M.u[q] + divide(M.b[q] - Au, dd);
}

// The same update as tail_sweep_cell (the same terms summed in the same order) for a run of
// sweeps of one small level by one warp: each lane's cell of a colour, its neighbours'
// shared indices (16 bits each: a shared image of at most 200 KB holds fewer than 2^16
// cells) and the operands that the sweeps do not change (diagonal, b, face coefficients)
// are gathered once into shared memory, so that a sweep is seven loads of u, the sum and
// the store.  (The compiler may pair products and additions into FMAs differently in the
// two forms, so they agree to FP32 rounding, not bit for bit.)
template <class TV>
struct TailCell {
    int qh;           // shared index | has << 16 (bit a: the neighbouring octet across axis a exists)
    int nb[3];        // per axis: partner index << 16 | neighbouring octet's cell (q when absent)
    TV dd, bq, cp[3], co[3];
};

template <class TV>
__device__ __forceinline__ void tail_cell_gather(const TailMem<TV>& M, const TailLevel& L, int colour, int i,
                                                 TailCell<TV>& C) {
    const int ni = L.ni, no = ni * ni * ni;
    const bool p2 = (no & (no - 1)) == 0;
    const int sh = p2 ? __ffs(no) - 1 : 0;
    const int k = p2 ? (i >> sh) : i / no;
    const int o = i - k * no;
    const int s = 2 * k + ((__popc(k) & 1) ^ colour);
    const int q = L.sbase + s * no + o;
    int crd[3];
    octet_coords(o, ni, crd[0], crd[1], crd[2]);
    const int stride[3] = {1, ni, ni * ni};
    int has = 0;
    C.dd = M.d[q];
    C.bq = M.b[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const int qi = L.sbase + (s ^ bit) * no + o;
        const bool up = (s & bit) != 0;
        const bool h = up ? crd[a] < ni - 1 : crd[a] > 0;
        const int qn = h ? (up ? qi + stride[a] : qi - stride[a]) : q;
        C.nb[a] = (qi << 16) | qn;
        C.cp[a] = M.cm[a][up ? q : qi];
        C.co[a] = M.cm[a][up ? qn : q];
        has |= h ? bit : 0;
    }
    C.qh = q | (has << 16);
}

template <class TV>
__device__ __forceinline__ void tail_cell_update(const TailMem<TV>& M, const TailCell<TV>& C) {
    const int q = C.qh & 0xffff;
    const TV uq = M.u[q];
    TV vp[3], vo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { vp[a] = M.u[C.nb[a] >> 16]; vo[a] = M.u[C.nb[a] & 0xffff]; }
    if (C.dd == TV(0)) return;
    TV Au = C.dd * uq;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Au += C.cp[a] * vp[a];
        if ((C.qh >> (16 + a)) & 1) Au += C.co[a] * vo[a];
    }
    M.u[q] = uq + divide(C.bq - Au, C.dd);
}

template <class TV>
__device__ __forceinline__ void tail_sweep_cells(const TailMem<TV>& M, const TailLevel& L, int colour) {
    const int no = L.ni * L.ni * L.ni;
    for (int i = threadIdx.x; i < 4 * no; i += blockDim.x) tail_sweep_cell<TV>(M, L, colour, i);
    __syncthreads();
}

// One pass over the octets of tail level li (li + 1 = the next coarser tail level, for
// restriction and prolongation).
template <class TV>
__device__ __forceinline__ void tail_pass(const TailMem<TV>& M, const TailArgs& A, int li, int kind, TV scale) {
    const TailLevel& L = A.L[li];
    const int no = tail_noct(L);
    for (int o = threadIdx.x; o < no; o += blockDim.x) {
        const int c0 = L.sbase + o;
        TV u[8], d[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) { u[s] = M.u[c0 + s * no]; d[s] = M.d[c0 + s * no]; }
        TV mean = TV(0);
        int n = 0;
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (d[s] != TV(0)) { mean += u[s]; ++n; }
        mean = mean * inv_count<TV>(n);
        if (kind == TP_PROLONG) {
            const TV uP = M.u[tail_parent(L, A.L[li + 1], o)];
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (d[s] != TV(0)) M.u[c0 + s * no] = u[s] + (uP - mean);
            continue;
        }
        TV cm[3][8], Au[8];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int s = 0; s < 8; ++s) cm[a][s] = M.cm[a][c0 + s * no];
        tail_octet_Au<TV>(M, L, o, u, d, cm, Au);
        if (kind == TP_FIXB) {
            // every real cell of a level m < 0 has children; padding cells are inactive
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (d[s] != TV(0)) M.b[c0 + s * no] += Au[s];
        } else if (kind == TP_RESTRICT) {
            TV rs = TV(0);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (d[s] != TV(0)) rs += M.b[c0 + s * no] - Au[s];
            const int P = tail_parent(L, A.L[li + 1], o);
            M.b[P] = scale * rs;
            M.u[P] = mean;
        } else {
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (((__popc(s) & 1) == kind) && d[s] != TV(0))
                    M.u[c0 + s * no] = u[s] + divide(M.b[c0 + s * no] - Au[s], d[s]);
        }
    }
    __syncthreads();
}

// The sub-cycle of Alg. 4 over the tail levels is expanded on the host into a flat
// schedule of passes (no recursion on the device); fas adds the FAS right-hand-side pass
// on the top tail level first.
template <class TV, class TC, class TW>
__device__ __forceinline__ void tail_cycle(const TailArgs& A, int fas, int prolong, const Tables& T,
                                           const Coefs<TC, TW>& C, TV* __restrict__ U, TV* __restrict__ B,
                                           TV scale) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = A.ncell;
    TailMem<TV> M;
    TV* base = reinterpret_cast<TV*>(smem);
    M.u = base; M.b = base + N; M.d = base + 2 * N;
    M.cm[0] = base + 3 * N; M.cm[1] = base + 4 * N; M.cm[2] = base + 5 * N;
    __shared__ int ssched[TAIL_SCHED_SH];
    __shared__ TailCell<TV> wcell[2][32];   // the warp-run sweeps' per-lane records, per colour
    const bool sch_sh = A.nsched <= TAIL_SCHED_SH;
    if (sch_sh)
        for (int q = threadIdx.x; q < A.nsched; q += blockDim.x) ssched[q] = A.sched[q];
    // global cell off + 8 o + s  <->  shared sbase + s * no + o; one octet per thread, so
    // that its vector loads of all six arrays are in flight together
    for (int li = 0; li < A.nlev; ++li) {
        const TailLevel& L = A.L[li];
        const int no = tail_noct(L);
        for (int o = threadIdx.x; o < no; o += blockDim.x) {
            const int g8 = L.off + 8 * o, q0 = L.sbase + o;
            TV u[8], b[8], d[8], cx[8], cy[8], cz[8];
            ldv8<true>(U, g8, u);
            ldv8<true>(B, g8, b);
            ldc8(C.d + g8, d);
            ldc8(C.cx + g8, cx);
            ldc8(C.cy + g8, cy);
            ldc8(C.cz + g8, cz);
#pragma unroll
            for (int sl = 0; sl < 8; ++sl) {
                const int q = q0 + sl * no;
                M.u[q] = u[sl]; M.b[q] = b[sl]; M.d[q] = d[sl];
                M.cm[0][q] = cx[sl]; M.cm[1][q] = cy[sl]; M.cm[2][q] = cz[sl];
            }
        }
    }
    __syncthreads();
    if (fas) tail_pass<TV>(M, A, 0, TP_FIXB, TV(0));
    for (int q = 0; q < A.nsched; ++q) {
        const int e = sch_sh ? ssched[q] : __ldg(A.sched + q);
        const int li = e >> 3, kind = e & 7;
        if (kind <= TP_SWEEP1 && 4 * tail_noct(A.L[li]) <= 32) {
            // a run of sweeps of a level whose colour has at most 32 cells (the coarsest):
            // the first warp does all of them, one cell per lane, ordered by warp barriers
            int q2 = q + 1;
            for (; q2 < A.nsched; ++q2) {
                const int e2 = sch_sh ? ssched[q2] : __ldg(A.sched + q2);
                if ((e2 >> 3) != li || (e2 & 7) > TP_SWEEP1) break;
            }
            if (threadIdx.x < 32) {
                const bool act = (int)threadIdx.x < 4 * tail_noct(A.L[li]);
                if (act) {
                    tail_cell_gather<TV>(M, A.L[li], 0, threadIdx.x, wcell[0][threadIdx.x]);
                    tail_cell_gather<TV>(M, A.L[li], 1, threadIdx.x, wcell[1][threadIdx.x]);
                }
                for (int k = q; k < q2; ++k) {
                    const int ek = sch_sh ? ssched[k] : __ldg(A.sched + k);
                    if (act) tail_cell_update<TV>(M, wcell[ek & 1][threadIdx.x]);
                    __syncwarp();
                }
            }
            __syncthreads();
            q = q2 - 1;
            continue;
        }
        if (kind <= TP_SWEEP1) tail_sweep_cells<TV>(M, A.L[li], kind);
        else tail_pass<TV>(M, A, li, kind, scale);
    }
    for (int li = 0; li < A.nlev; ++li) {
        const TailLevel& L = A.L[li];
        const int no = tail_noct(L);
        for (int o = threadIdx.x; o < no; o += blockDim.x) {
            TV u[8], b[8];
#pragma unroll
            for (int sl = 0; sl < 8; ++sl) { u[sl] = M.u[L.sbase + sl * no + o]; b[sl] = M.b[L.sbase + sl * no + o]; }
            stv8<true>(U, L.off + 8 * o, u);
            stv8<true>(B, L.off + 8 * o, b);
        }
    }
    if (prolong) {
        // onto the level above the tail, one child octet per thread: child octet (I, J, K)
        // of that uniform level has the parent cell (I, J, K) of the top tail level
        const TailLevel& L = A.L[0];
        const int no = tail_noct(L), nu = A.up_ni;
        const int nco = nu * nu * nu;
        for (int co = threadIdx.x; co < nco; co += blockDim.x) {
            int I, J, K;
            octet_coords(co, nu, I, J, K);
            const int po = (I >> 1) + L.ni * ((J >> 1) + L.ni * (K >> 1));
            const int sl = (I & 1) | ((J & 1) << 1) | ((K & 1) << 2);
            octet_prolong<TV>(C.d, U, A.up_off / 8 + co, M.u[L.sbase + sl * no + po]);
        }
    }
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(sizeof(TV) == 8 ? 256 : 1024)
    k_otail(TailArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U, TV* __restrict__ B, TV scale) {
    pdl_enter();
    tail_cycle<TV, TC, TW>(A, A.fas, A.prolong, T, C, U, B, scale);
}

}  // namespace ocg
