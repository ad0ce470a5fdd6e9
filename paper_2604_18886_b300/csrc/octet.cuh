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

template <class TV>
struct OctState {
    TV u[8], d[8], cm[3][8];
    TV ubar;      // mean of the active cells
    int nact;
};

// Loads u and the coefficients of the octet whose first cell is c8.
template <class TV, class TC, class TW>
__device__ __forceinline__ void load_octet(const TV* __restrict__ U, const Coefs<TC, TW>& C, int c8,
                                           OctState<TV>& S) {
    ld8(U + c8, S.u);
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
    S.ubar = n ? s / TV(n) : TV(0);
}

// Au[s] = (A^m u) for the 8 cells of octet o (global index og) of the level starting at
// cell `off`; U is read for the neighbouring octets and the coarser leaves K.
template <class TV, class TC, class TW>
__device__ __forceinline__ void octet_Au(const Tables& T, const Coefs<TC, TW>& C, const TV* __restrict__ U, int off,
                                         int og, const OctState<TV>& S, TV (&Au)[8]) {
#pragma unroll
    for (int s = 0; s < 8; ++s) Au[s] = S.d[s] * S.u[s];
    int nb[6];
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) nb[dir] = __ldg(T.nbr + dir * T.noct + og);
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
#pragma unroll
            for (int q = 0; q < 4; ++q) nu[q] = U[n8 + (clear_slot(a, q) | bit)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += S.cm[a][s] * nu[q];
            }
        } else if (v <= -2) {
            const int t = -2 - v;
            const TV uK = U[__ldg(T.tK + (2 * a) * T.nt + t)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q);
                Au[s] += S.cm[a][s] * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
        // + face: cells with bit set meet the - side of the + neighbour, whose cells keep
        // the face coefficients
        const int w = nb[2 * a + 1];
        if (w >= 0) {
            const int n8 = off + 8 * w;
            const TC* cc = a == 0 ? C.cx : (a == 1 ? C.cy : C.cz);
            TV nu[4], nc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                nu[q] = U[n8 + clear_slot(a, q)];
                nc[q] = TV(tov(__ldg(cc + n8 + clear_slot(a, q))));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) Au[clear_slot(a, q) | bit] += nc[q] * nu[q];
        } else if (w <= -2) {
            const int t = -2 - w;
            const TV uK = U[__ldg(T.tK + (2 * a + 1) * T.nt + t)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = clear_slot(a, q) | bit;
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + q) * T.nt + t)));
                Au[s] += cf * (S.u[s] + (uK - S.ubar) * TV(0.5));
            }
        }
    }
}

template <class TV, class TC>
__device__ __forceinline__ void octet_prolong(const TC* __restrict__ d, TV* __restrict__ U, int co, TV uP) {
    const int c8 = 8 * co;
    TV v[8], dd[8];
    ld8(U + c8, v);
    ldc8(d + c8, dd);
    TV s = TV(0);
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != TV(0)) { s += v[q]; ++n; }
    if (n == 0) return;
    const TV delta = uP - s / TV(n);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != TV(0)) U[c8 + q] = v[q] + delta;
}

// Red-black colour sweep (Sec. 2.3) of a level, or (fixb) completion of the FAS
// right-hand side b += A^m u* on cells with children (Alg. 4).  prolong: after the
// update, every cell with children prolongs its final value onto them.
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_osweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                 TV* __restrict__ B, int colour, int prolong, int fixb) {
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    const int og = c8 >> 3;
    OctState<TV> S;
    load_octet<TV, TC, TW>(U, C, c8, S);
    octet_mean(S);
    TV b[8], Au[8];
    ld8(B + c8, b);
    octet_Au<TV, TC, TW>(T, C, U, A.off, og, S, Au);
    if (fixb) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (__ldg(T.child_oct + c8 + s) >= 0) B[c8 + s] = b[s] + Au[s];
        return;
    }
    TV un[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        un[s] = S.u[s];
        if (((__popc(s) & 1) == colour) && S.d[s] != TV(0)) {
            un[s] = S.u[s] + (b[s] - Au[s]) / S.d[s];
            U[c8 + s] = un[s];
        }
    }
    if (prolong) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int co = __ldg(T.child_oct + c8 + s);
            if (co >= 0) octet_prolong<TV, TC>(C.d, U, co, un[s]);
        }
    }
}

// Residual and FAS restriction (Alg. 4): r = b - A^m u; the parent gets
// b_P = (beta/alpha) sum r (A^{m-1} u* is added on the coarse level by the fixb pass) and
// u_P = u* = mean of the active children.
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_orestrict(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                    TV* __restrict__ B, TV scale) {
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    const int og = c8 >> 3;
    OctState<TV> S;
    load_octet<TV, TC, TW>(U, C, c8, S);
    octet_mean(S);
    TV b[8], Au[8];
    ld8(B + c8, b);
    octet_Au<TV, TC, TW>(T, C, U, A.off, og, S, Au);
    TV rs = TV(0);
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (S.d[s] != TV(0)) rs += b[s] - Au[s];
    const int P = __ldg(T.oct_parent + og);
    B[P] = scale * rs;
    U[P] = S.ubar;
}

// Prolongation as its own launch (thread per child octet).
template <class TV, class TC>
__global__ void __launch_bounds__(OBLK) k_oprolong(LevelArgs A, Tables T, const TC* __restrict__ d,
                                                   TV* __restrict__ U) {
    const int o = blockIdx.x * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    octet_prolong<TV, TC>(d, U, c8 >> 3, U[__ldg(T.oct_parent + (c8 >> 3))]);
}

// Outer vector: parent value = mean of the active children (composite operator, Sec. 3.1).
template <class TO, class TC>
__global__ void __launch_bounds__(OBLK) k_oavg(LevelArgs A, Tables T, const TC* __restrict__ d, TO* __restrict__ P) {
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
    P[__ldg(T.oct_parent + (c8 >> 3))] = n ? s / TO(n) : TO(0);
}

// Composite leaf operator over all tree levels in one launch (block -> level lookup):
// Y = A p on leaves, 0 on inner cells; (p, A p) over leaves reduced into R.
struct OMultiLevel {
    int n;
    int off[MAXLEV];
    int noct[MAXLEV];
    int boff[MAXLEV + 1];
};

template <class TO, class TC, class TW>
__global__ void __launch_bounds__(OBLK) k_oapply(OMultiLevel ML, Tables T, Coefs<TC, TW> C, const TO* __restrict__ P,
                                                 TO* __restrict__ Y, Red R) {
    __shared__ double sh[32];
    int l = 0;
    while (l + 1 < ML.n && (int)blockIdx.x >= ML.boff[l + 1]) ++l;
    const int o = ((int)blockIdx.x - ML.boff[l]) * OBLK + threadIdx.x;
    double dot = 0.0;
    if (o < ML.noct[l]) {
        const int c8 = ML.off[l] + 8 * o;
        OctState<TO> S;
        load_octet<TO, TC, TW>(P, C, c8, S);
        octet_mean(S);
        TO Ap[8];
        octet_Au<TO, TC, TW>(T, C, P, ML.off[l], c8 >> 3, S, Ap);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const bool leaf = __ldg(T.child_oct + c8 + s) < 0;
            Y[c8 + s] = leaf ? Ap[s] : TO(0);
            if (leaf) dot += (double)S.u[s] * (double)Ap[s];
        }
    }
    if (R.op != OP_NONE) red_finish(R, blockIdx.x, dot, 0.0, sh);
}

}  // namespace ocg
