// libocg device kernels (sm_103a).
//
// Thread mapping: one thread per cell; the 8 cells of an octet (children of one coarse
// cell, slot s = dx + 2 dy + 4 dz) sit in 8 consecutive lanes.  Within an octet the
// face neighbour along axis a is slot s ^ (1 << a) and is read with a warp shuffle;
// the neighbour across the octet boundary is slot s ^ (1 << a) of the neighbouring
// octet (table nbr).  The T-junction ghost needs the mean of the 8 siblings
// (Sec. 3.1, pbar_P), which is a 3-step shuffle reduction over the octet's lanes, and
// the value of the coarser leaf K (record tK).  No tensor cores: the operator is a
// 7-point stencil, bound by memory traffic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLK = 256;

struct Tables {
    const int32_t* nbr;        // [6][noct] level-local octet / -1 wall / -2-t T record
    const int32_t* oct_parent; // [noct] global parent cell
    const int32_t* child_oct;  // [ncell] global children octet or -1
    const int32_t* tK;         // [6][nt]
    int64_t noct;
    int64_t nt;
};

struct LevelArgs {
    int64_t off;      // first global cell of the level
    int64_t ncell;    // multiple of 8
};

template <class TC, class TW>
struct Coefs {
    const TC* d;
    const TC* cx;
    const TC* cy;
    const TC* cz;
    const TW* tw;     // [24][nt]: coefficient (-w_f) of each fine T face, slot (dir*4+q)
};

__device__ __forceinline__ double tov(double v) { return v; }
__device__ __forceinline__ float tov(float v) { return v; }
__device__ __forceinline__ float tov(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int sub_index(int a, int s) {
    return a == 0 ? (((s >> 1) & 1) | (((s >> 2) & 1) << 1))
         : a == 1 ? ((s & 1) | (((s >> 2) & 1) << 1))
                  : ((s & 1) | (((s >> 1) & 1) << 1));
}

template <class TC, class TW>
__device__ __forceinline__ TC coef_axis(const Coefs<TC, TW>& C, int a, int64_t g) {
    return a == 0 ? C.cx[g] : (a == 1 ? C.cy[g] : C.cz[g]);
}

// Sum over the 8 lanes of the calling thread's octet.
template <class T>
__device__ __forceinline__ T octet_sum(T v) {
    v += __shfl_xor_sync(FULL, v, 1);
    v += __shfl_xor_sync(FULL, v, 2);
    v += __shfl_xor_sync(FULL, v, 4);
    return v;
}

// Mean of the active cells (c != 0) of the octet; 0 when none is active.
template <class TV>
__device__ __forceinline__ TV octet_active_mean(TV u, bool act) {
    const TV s = octet_sum<TV>(act ? u : TV(0));
    const unsigned bal = __ballot_sync(FULL, act);
    const int cnt = __popc((bal >> (threadIdx.x & 24)) & 0xffu);
    return cnt ? s / TV(cnt) : TV(0);
}

// (A^m u)_g for the cell in slot s of global octet og of a level starting at `off`:
// c u + sum over faces of c_face u_nb, c_face the stored coefficient of the face (kept
// by its + cell).  A T face (neighbour region covered by a coarser leaf K) uses the
// ghost g = u + (u_K - ubar)/2 (Sec. 3.1, Eq. t-junction-ghost-values).
// Must be called by all 32 lanes of the warp (shuffles).
template <class TV, class TC, class TW>
__device__ __forceinline__ TV stencil_Au(const Tables& T, const Coefs<TC, TW>& C, const TV* __restrict__ U,
                                         int64_t off, int64_t og, int s, TV u, TV ubar, TV dd,
                                         const TV cm[3]) {
    TV Au = dd * u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const TV ca = cm[a];
        const TV u_in = __shfl_xor_sync(FULL, u, bit);
        const TV ca_in = __shfl_xor_sync(FULL, ca, bit);
        if (s & bit) {
            Au += ca * u_in;                                  // face towards slot s^bit
            const int v = T.nbr[(int64_t)(2 * a + 1) * T.noct + og];
            if (v >= 0) {
                const int64_t ng = off + 8 * (int64_t)v + (s ^ bit);
                Au += TV(tov(coef_axis(C, a, ng))) * U[ng];
            } else if (v <= -2) {
                const int64_t t = -2 - v;
                const int64_t K = T.tK[(int64_t)(2 * a + 1) * T.nt + t];
                const TV cf = TV(tov(C.tw[(int64_t)((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + t]));
                Au += cf * (u + (U[K] - ubar) * TV(0.5));
            }
        } else {
            Au += ca_in * u_in;
            const int v = T.nbr[(int64_t)(2 * a) * T.noct + og];
            if (v >= 0) {
                const int64_t ng = off + 8 * (int64_t)v + (s ^ bit);
                Au += ca * U[ng];
            } else if (v <= -2) {
                const int64_t t = -2 - v;
                const int64_t K = T.tK[(int64_t)(2 * a) * T.nt + t];
                Au += ca * (u + (U[K] - ubar) * TV(0.5));
            }
        }
    }
    return Au;
}

enum { MODE_SWEEP = 0, MODE_FIXB = 2 };

// One red-black Gauss-Seidel colour sweep of level m (Sec. 2.3): cells of `colour`
// ((i+j+k) mod 2 = popcount(s) mod 2, octet bases are even) get u += (b - A u)/c from
// the state at the start of the sweep: a cell of `colour` reads only cells of the other
// colour, the coarser leaf of a T ghost, and its own octet's values loaded before any
// store, so no value it reads changes during the launch.
// MODE_FIXB instead completes the FAS right-hand side of cells with children,
// b = beta R r + A^{m} u* (Alg. 4), and updates nothing; it runs as its own launch
// because every cell must see the unmodified state.
template <class TV, class TC, class TW, int MODE>
__global__ void __launch_bounds__(BLK) k_sweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                               TV* __restrict__ B, int colour) {
    const int64_t tid = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int64_t g = A.off + lc;
    const int s = (int)(lc & 7);
    const int64_t og = g >> 3;
    const TV u = U[g];
    TV b = B[g];
    const TV dd = TV(tov(C.d[g]));
    const TV cm[3] = {TV(tov(C.cx[g])), TV(tov(C.cy[g])), TV(tov(C.cz[g]))};
    const bool act = dd != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    const TV Au = stencil_Au<TV, TC, TW>(T, C, U, A.off, og, s, u, ubar, dd, cm);
    if (MODE == MODE_FIXB) {
        if (valid && T.child_oct[g] >= 0) B[g] = b + Au;
    } else {
        if (valid && act && ((__popc(s) & 1) == colour)) U[g] = u + (b - Au) / dd;
    }
}

// Residual and FAS restriction from level m to its parents (Alg. 4): r = b - A^m u,
// u*_P = mean of the active children, b_P = (beta/alpha) sum_children r (the A^{m-1} u*
// term is added on the coarse level by a MODE_FIXB launch).
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_restrict(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                  TV* __restrict__ B, TV scale) {
    const int64_t tid = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int64_t g = A.off + lc;
    const int s = (int)(lc & 7);
    const int64_t og = g >> 3;
    const TV u = U[g];
    const TV b = B[g];
    const TV dd = TV(tov(C.d[g]));
    const TV cm[3] = {TV(tov(C.cx[g])), TV(tov(C.cy[g])), TV(tov(C.cz[g]))};
    const bool act = dd != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    const TV Au = stencil_Au<TV, TC, TW>(T, C, U, A.off, og, s, u, ubar, dd, cm);
    const TV r = act ? b - Au : TV(0);
    const TV rs = octet_sum<TV>(r);
    if (valid && s == 0) {
        const int64_t P = T.oct_parent[og];
        B[P] = scale * rs;
        U[P] = ubar;
    }
}

// Prolongation (Alg. 4): u += u_P - u*_P on the active children, u* = Avg(children),
// which is still the children's mean because level m is untouched since restriction.
template <class TV, class TC>
__global__ void __launch_bounds__(BLK) k_prolong(LevelArgs A, Tables T, const TC* __restrict__ d,
                                                 TV* __restrict__ U) {
    const int64_t tid = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int64_t g = A.off + lc;
    const int64_t og = g >> 3;
    const TV u = U[g];
    const bool act = TV(tov(d[g])) != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    if (valid && act) U[g] = u + (U[T.oct_parent[og]] - ubar);
}

// Coarsest level (one CTA): nu sweeps, half red->black then half black->red; with
// fas != 0 the FAS right-hand side of cells with children is completed first.
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(1024) k_coarsest(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                   TV* __restrict__ B, int nu, int fas) {
    const int nb = blockDim.x;
    auto pass = [&](int colour, int mode) {
        for (int64_t base = 0; base < A.ncell; base += nb) {
            const int64_t tid = base + threadIdx.x;
            const bool valid = tid < A.ncell;
            const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
            const int64_t g = A.off + lc;
            const int s = (int)(lc & 7);
            const TV u = U[g];
            TV b = B[g];
            const TV dd = TV(tov(C.d[g]));
            const TV cm[3] = {TV(tov(C.cx[g])), TV(tov(C.cy[g])), TV(tov(C.cz[g]))};
            const bool act = dd != TV(0);
            const TV ubar = octet_active_mean<TV>(u, act);
            const TV Au = stencil_Au<TV, TC, TW>(T, C, U, A.off, g >> 3, s, u, ubar, dd, cm);
            if (mode == MODE_FIXB) {
                if (valid && T.child_oct[g] >= 0) B[g] = b + Au;
            } else if (valid && act && ((__popc(s) & 1) == colour)) {
                U[g] = u + (b - Au) / dd;
            }
        }
        __syncthreads();
    };
    if (fas) pass(0, MODE_FIXB);
    const int half = nu / 2;
    for (int it = 0; it < half; ++it) { pass(0, MODE_SWEEP); pass(1, MODE_SWEEP); }
    for (int it = half; it < nu; ++it) { pass(1, MODE_SWEEP); pass(0, MODE_SWEEP); }
}

// Inner values of the outer vector: p_P = mean of P's active children (level m cells
// -> parents at level m-1), used by the composite operator (pbar_P and the coarse side).
template <class TO, class TC>
__global__ void __launch_bounds__(BLK) k_avg(LevelArgs A, Tables T, const TC* __restrict__ d, TO* __restrict__ P) {
    const int64_t tid = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int64_t g = A.off + lc;
    const TO u = P[g];
    const bool act = TO(tov(d[g])) != TO(0);
    const TO m = octet_active_mean<TO>(u, act);
    if (valid && (lc & 7) == 0) P[T.oct_parent[g >> 3]] = m;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    }
    return t;  // valid in thread 0
}

// Composite leaf operator on one tree level: Y = A p on leaves, 0 on inner cells; the
// block partials of (p, A p) over leaves go to part[blockIdx.x].
template <class TO, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_apply(LevelArgs A, Tables T, Coefs<TC, TW> C, const TO* __restrict__ P,
                                               TO* __restrict__ Y, double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t tid = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int64_t lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int64_t g = A.off + lc;
    const int s = (int)(lc & 7);
    const TO p = P[g];
    const TO dd = TO(tov(C.d[g]));
    const TO cm[3] = {TO(tov(C.cx[g])), TO(tov(C.cy[g])), TO(tov(C.cz[g]))};
    const bool act = dd != TO(0);
    const TO pbar = octet_active_mean<TO>(p, act);
    const TO Ap = stencil_Au<TO, TC, TW>(T, C, P, A.off, g >> 3, s, p, pbar, dd, cm);
    const bool leaf = T.child_oct[g] < 0;
    const TO y = leaf ? Ap : TO(0);
    if (valid) Y[g] = y;
    if (part) {
        const double v = (valid && leaf) ? (double)p * (double)Ap : 0.0;
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// ----------------------------------------------------------------- PCG vector kernels
template <class TI, class TO>
__global__ void k_scatter(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                          int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[leaf_cell[r]] = TO(in[r]);
}

template <class TI, class TO>
__global__ void k_gather(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                         int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = TO(in[leaf_cell[r]]);
}

enum { S_PAP = 0, S_ALPHA, S_RZ, S_BETA, S_RR, S_RS, S_MEAN, S_BB, S_RR0, S_NS, S_COUNT = 16 };

// x += alpha p, r -= alpha Ap over the tree cells; partial sums of r.r and sum(r)
// (inner cells keep r = 0 since Ap = 0 there); optionally b32 = r.
template <class TO, class TB>
__global__ void __launch_bounds__(BLK) k_update(TO* __restrict__ x, TO* __restrict__ r, const TO* __restrict__ p,
                                                const TO* __restrict__ Ap, const double* __restrict__ S,
                                                TB* __restrict__ b32, int64_t n, double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    const double alpha = S[S_ALPHA];
    double rr = 0.0, rs = 0.0;
    if (i < n) {
        x[i] = x[i] + TO(alpha) * p[i];
        const TO rn = r[i] - TO(alpha) * Ap[i];
        r[i] = rn;
        if (b32) b32[i] = TB(rn);
        rr = (double)rn * (double)rn;
        rs = (double)rn;
    }
    const double t1 = block_sum(rr, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t1;
    const double t2 = block_sum(rs, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t2;
}

// r -= mean on leaves (null-space shift of Sec. 2.2) and b32 = r.
template <class TO, class TB>
__global__ void k_project(TO* __restrict__ r, const uint8_t* __restrict__ flags, const double* __restrict__ S,
                          TB* __restrict__ b32, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TO v = r[i];
    if (flags[i] & 1) v = v - TO(S[S_MEAN]);
    r[i] = v;
    if (b32) b32[i] = TB(v);
}

// partial sums of (a, b) and of a (for the mean) over the first n cells
template <class TA, class TB>
__global__ void __launch_bounds__(BLK) k_dot(const TA* __restrict__ a, const TB* __restrict__ b, int64_t n,
                                             double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    double v = 0.0, s = 0.0;
    if (i < n) {
        v = (double)a[i] * (double)b[i];
        s = (double)a[i];
    }
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    const double t2 = block_sum(s, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t2;
}

// residual partials: (b - y) over leaves, for the true residual at exit
template <class TO>
__global__ void __launch_bounds__(BLK) k_resid(const TO* __restrict__ b, const TO* __restrict__ y,
                                               const uint8_t* __restrict__ flags, int64_t n, double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t i = blockIdx.x * (int64_t)BLK + threadIdx.x;
    double v = 0.0, s = 0.0;
    if (i < n && (flags[i] & 1)) {
        const double d = (double)b[i] - (double)y[i];
        v = d * d;
        s = d;
    }
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    const double t2 = block_sum(s, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t2;
}

template <class TO, class TZ>
__global__ void k_pupdate(TO* __restrict__ p, const TZ* __restrict__ z, const double* __restrict__ S, int64_t n,
                          int first) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = first ? TO(z[i]) : TO(z[i]) + TO(S[S_BETA]) * p[i];
}

enum { OP_ALPHA = 0, OP_RR = 1, OP_BETA = 2, OP_RZ0 = 3, OP_BB = 4, OP_MEAN = 5 };

// Fixed-order reduction of nb block partials (two rows for OP_RR / OP_BB / OP_MEAN) and
// the scalar step of Alg. 1 (alpha, beta) on the device.
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ part, int64_t nb, int op,
                                                  double* __restrict__ S, double nleaf) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
    const bool two = (op == OP_RR || op == OP_BB || op == OP_MEAN);
    if (two)
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) b += part[nb + i];
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    if (threadIdx.x != 0) return;
    const bool ns = S[S_NS] != 0.0;
    switch (op) {
        case OP_ALPHA: S[S_PAP] = sa; S[S_ALPHA] = S[S_RZ] / sa; break;
        case OP_RZ0: S[S_RZ] = sa; break;
        case OP_BETA: S[S_BETA] = sa / S[S_RZ]; S[S_RZ] = sa; break;
        case OP_RR:
        case OP_BB: {
            const double mean = ns ? sb / nleaf : 0.0;
            const double rr = ns ? sa - sb * mean : sa;
            S[S_MEAN] = mean;
            S[op == OP_RR ? S_RR : S_BB] = rr;
            break;
        }
        case OP_MEAN: S[S_MEAN] = ns ? sb / nleaf : 0.0; break;
    }
}

// ----------------------------------------------------------------- setup kernels (FP64)

// -beta_f h_f into the face's destination: the - face coefficient of its + cell, or the
// T record weight of a fine leaf's + face.  Flags a negative / non-finite beta.
__global__ void k_face_scatter(const float* __restrict__ beta, const int64_t* __restrict__ slot,
                               const uint8_t* __restrict__ kind, const int32_t* __restrict__ depth,
                               const double* __restrict__ hdepth, int64_t nface, double* __restrict__ cm,
                               double* __restrict__ tw, int* __restrict__ err) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nface) return;
    const float b = beta[f];
    if (!(b >= 0.0f) || !isfinite(b)) atomicOr(err, 1);
    const double w = (double)b * hdepth[depth[f]];
    if (kind[f] == 0) cm[slot[f]] = -w;
    else tw[slot[f]] = -w;
}

struct LevelTab {
    int64_t off[32];
    double h[32];
    int mc;
};

// Per leaf: the - face coefficients the scatter could not write (walls; coarse side of a
// T-junction = (1/2) sum of the fine sub-face weights, Sec. 3.1) and the diagonal = sum of
// the six face weights (Eq. projection-poisson-system).
__global__ void k_leaf_gather(const int32_t* __restrict__ leaf_cell, const int8_t* __restrict__ level,
                              Tables T, LevelTab LT, int4 bc_lo, int2 bc_hi, int64_t nleaf, int64_t ncell,
                              double* __restrict__ dg, double* __restrict__ cm, const double* __restrict__ tw) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nleaf) return;
    const int bc[6] = {bc_lo.x, bc_lo.y, bc_lo.z, bc_lo.w, bc_hi.x, bc_hi.y};
    const int64_t g = leaf_cell[r];
    const int m = level[g];
    const int64_t off = LT.off[m - LT.mc];
    const double h = LT.h[m - LT.mc];
    const int s = (int)((g - off) & 7);
    const int64_t og = g >> 3;
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        double* cma = cm + (int64_t)a * ncell;
        // - face
        double wm;
        int64_t nmi = -1;   // same-depth cell on the - side
        bool wall = false;
        if (s & bit) nmi = g ^ bit;
        else {
            const int v = T.nbr[(int64_t)(2 * a) * T.noct + og];
            if (v >= 0) nmi = off + 8 * (int64_t)v + (s ^ bit);
            else if (v == -1) wall = true;
        }
        if (wall) {
            wm = bc[2 * a] ? 2.0 * h : 0.0;
            cma[g] = -wm;
        } else if (nmi >= 0 && T.child_oct[nmi] >= 0) {
            // coarse side: children of nmi with bit a = 1 hold fine + faces in their T record
            const int64_t co = T.child_oct[nmi];
            const int v = T.nbr[(int64_t)(2 * a + 1) * T.noct + co];
            const int64_t t = -2 - v;
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) acc += tw[(int64_t)((2 * a + 1) * 4 + q) * T.nt + t];
            cma[g] = 0.5 * acc;
            wm = -0.5 * acc;
        } else {
            wm = -cma[g];   // regular or fine side of a T-junction (written by the scatter)
        }
        // + face
        double wp;
        int64_t npl = -1;
        wall = false;
        int tplus = -1;
        if (!(s & bit)) npl = g ^ bit;
        else {
            const int v = T.nbr[(int64_t)(2 * a + 1) * T.noct + og];
            if (v >= 0) npl = off + 8 * (int64_t)v + (s ^ bit);
            else if (v == -1) wall = true;
            else tplus = -2 - v;
        }
        if (wall) {
            wp = bc[2 * a + 1] ? 2.0 * h : 0.0;
        } else if (tplus >= 0) {
            wp = -tw[(int64_t)((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + tplus];
        } else if (T.child_oct[npl] >= 0) {
            // coarse side: the four children of npl with bit a = 0 keep the fine - faces
            const int64_t c8 = 8 * (int64_t)T.child_oct[npl];
            double acc = 0.0;
            for (int sl = 0; sl < 8; ++sl)
                if (!(sl & bit)) acc += cma[c8 + sl];
            wp = -0.5 * acc;
        } else {
            wp = -cma[npl];
        }
        diag += wm;
        diag += wp;
    }
    dg[g] = diag;
}

// Alg. 3 (Sec. 2.5) for the parent of each octet of level m: diagonal from the active
// children's diagonals / alpha plus (2/alpha) times the internal faces between active
// children; - face coefficients from the children on the parent's - faces / alpha.
__global__ void k_coarsen(LevelArgs A, Tables T, double alpha, double* __restrict__ dg, double* __restrict__ cm,
                          int64_t ncell) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int64_t c8 = A.off + 8 * o;
    const int64_t P = T.oct_parent[c8 >> 3];
    double c = 0.0, cxm[3] = {0.0, 0.0, 0.0};
    int active = 0;
    for (int s = 0; s < 8; ++s) {
        const double cc = dg[c8 + s];
        if (cc != 0.0) {
            ++active;
            c += cc / alpha;
        }
        for (int a = 0; a < 3; ++a) {
            const int bit = 1 << a;
            const double ca = cm[(int64_t)a * ncell + c8 + s];
            if (s & bit) {
                if (cc != 0.0 && dg[c8 + (s ^ bit)] != 0.0) c += (2.0 / alpha) * ca;
            } else {
                cxm[a] += ca / alpha;
            }
        }
    }
    if (active == 0) c = 0.0;
    dg[P] = c;
    for (int a = 0; a < 3; ++a) cm[(int64_t)a * ncell + P] = cxm[a];
}

template <class TS>
__global__ void k_convert(const double* __restrict__ in, TS* __restrict__ out, int64_t n);

template <>
__global__ void k_convert<float>(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

template <>
__global__ void k_convert<__nv_bfloat16>(const double* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn((float)in[i]);
}

}  // namespace ocg
