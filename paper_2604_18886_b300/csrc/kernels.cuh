// libocg device kernels (sm_103a).
//
// Thread mapping: one thread per cell; the 8 cells of an octet (children of one coarse
// cell, slot s = dx + 2 dy + 4 dz) sit in 8 consecutive lanes.  Within an octet the
// face neighbour along axis a is slot s ^ (1 << a) and is read with a warp shuffle;
// the neighbour across the octet boundary is slot s ^ (1 << a) of the neighbouring
// octet (table nbr).  The T-junction ghost needs the mean of the 8 siblings
// (Sec. 3.1, pbar_P), which is a 3-step shuffle reduction over the octet's lanes, and
// the value of the coarser leaf K (record tK).  No tensor cores: the operator is a
// 7-point stencil, bound by memory traffic and latency.  Cell indices fit in int32
// (the host rejects larger trees).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLK = 256;
constexpr int MAXLEV = 16;

struct Tables {
    const int32_t* nbr;        // [6][noct] level-local octet / -1 wall / -2-t T record
    const int32_t* oct_parent; // [noct] global parent cell
    const int32_t* child_oct;  // [ncell] global children octet or -1
    const int32_t* tK;         // [6][nt]
    int noct;
    int nt;
};

struct LevelArgs {
    int off;      // first global cell of the level
    int ncell;    // multiple of 8
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
__device__ __forceinline__ TC coef_axis(const Coefs<TC, TW>& C, int a, int g) {
    return a == 0 ? __ldg(C.cx + g) : (a == 1 ? __ldg(C.cy + g) : __ldg(C.cz + g));
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
                                         int off, int og, int s, TV u, TV ubar, TV dd, const TV cm[3]) {
    TV Au = dd * u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const TV ca = cm[a];
        const TV u_in = __shfl_xor_sync(FULL, u, bit);
        const TV ca_in = __shfl_xor_sync(FULL, ca, bit);
        if (s & bit) {
            Au += ca * u_in;                                  // face towards slot s^bit
            const int v = __ldg(T.nbr + (2 * a + 1) * T.noct + og);
            if (v >= 0) {
                const int ng = off + 8 * v + (s ^ bit);
                Au += TV(tov(coef_axis(C, a, ng))) * U[ng];
            } else if (v <= -2) {
                const int t = -2 - v;
                const int K = __ldg(T.tK + (2 * a + 1) * T.nt + t);
                const TV cf = TV(tov(__ldg(C.tw + ((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + t)));
                Au += cf * (u + (U[K] - ubar) * TV(0.5));
            }
        } else {
            Au += ca_in * u_in;
            const int v = __ldg(T.nbr + (2 * a) * T.noct + og);
            if (v >= 0) {
                const int ng = off + 8 * v + (s ^ bit);
                Au += ca * U[ng];
            } else if (v <= -2) {
                const int t = -2 - v;
                const int K = __ldg(T.tK + (2 * a) * T.nt + t);
                Au += ca * (u + (U[K] - ubar) * TV(0.5));
            }
        }
    }
    return Au;
}

// Prolongation of one parent onto its children octet (Alg. 4): u_c += u_P - u*_P on the
// active children, u* = mean of the active children (unchanged since restriction).
template <class TV, class TC>
__device__ __forceinline__ void prolong_children(const TC* __restrict__ d, TV* __restrict__ U, int co, TV uP) {
    const int c8 = 8 * co;
    TV v[8];
    bool act[8];
    TV s = TV(0);
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        v[q] = U[c8 + q];
        act[q] = tov(__ldg(d + c8 + q)) != 0;
        if (act[q]) { s += v[q]; ++n; }
    }
    if (n == 0) return;
    const TV delta = uP - s / TV(n);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (act[q]) U[c8 + q] = v[q] + delta;
}

enum { MODE_SWEEP = 0, MODE_FIXB = 2 };

// One red-black Gauss-Seidel colour sweep of level m (Sec. 2.3): cells of `colour`
// ((i+j+k) mod 2 = popcount(s) mod 2, octet bases are even) get u += (b - A u)/c from
// the state at the start of the sweep: a cell of `colour` reads only cells of the other
// colour, the coarser leaf of a T ghost, and its own octet's values loaded before any
// store, so no value it reads changes during the launch.
// With prolong != 0 (last post-smoothing sweep of a visit), every cell with children
// then prolongs its final value onto them (the finer level is not read by this launch).
// MODE_FIXB instead completes the FAS right-hand side of cells with children,
// b = beta R r + A^{m} u* (Alg. 4), and updates nothing; it runs as its own launch
// because every cell must see the unmodified state.
template <class TV, class TC, class TW, int MODE>
__global__ void __launch_bounds__(BLK) k_sweep(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                               TV* __restrict__ B, int colour, int prolong) {
    const int tid = blockIdx.x * BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int g = A.off + lc;
    const int s = lc & 7;
    const int og = g >> 3;
    const TV u = U[g];
    const TV b = B[g];
    const TV dd = TV(tov(__ldg(C.d + g)));
    const TV cm[3] = {TV(tov(__ldg(C.cx + g))), TV(tov(__ldg(C.cy + g))), TV(tov(__ldg(C.cz + g)))};
    const bool act = dd != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    const TV Au = stencil_Au<TV, TC, TW>(T, C, U, A.off, og, s, u, ubar, dd, cm);
    if (MODE == MODE_FIXB) {
        if (valid && __ldg(T.child_oct + g) >= 0) B[g] = b + Au;
    } else {
        TV un = u;
        if (valid && act && ((__popc(s) & 1) == colour)) {
            un = u + (b - Au) / dd;
            U[g] = un;
        }
        if (prolong && valid) {
            const int co = __ldg(T.child_oct + g);
            if (co >= 0) prolong_children<TV, TC>(C.d, U, co, un);
        }
    }
}

// Residual and FAS restriction from level m to its parents (Alg. 4): r = b - A^m u,
// u*_P = mean of the active children, b_P = (beta/alpha) sum_children r (the A^{m-1} u*
// term is added on the coarse level by a MODE_FIXB launch).
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_restrict(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                  TV* __restrict__ B, TV scale) {
    const int tid = blockIdx.x * BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int g = A.off + lc;
    const int s = lc & 7;
    const int og = g >> 3;
    const TV u = U[g];
    const TV b = B[g];
    const TV dd = TV(tov(__ldg(C.d + g)));
    const TV cm[3] = {TV(tov(__ldg(C.cx + g))), TV(tov(__ldg(C.cy + g))), TV(tov(__ldg(C.cz + g)))};
    const bool act = dd != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    const TV Au = stencil_Au<TV, TC, TW>(T, C, U, A.off, og, s, u, ubar, dd, cm);
    const TV r = act ? b - Au : TV(0);
    const TV rs = octet_sum<TV>(r);
    if (valid && s == 0) {
        const int P = __ldg(T.oct_parent + og);
        B[P] = scale * rs;
        U[P] = ubar;
    }
}

// Prolongation as its own launch (used when the coarse level cannot fuse it).
template <class TV, class TC>
__global__ void __launch_bounds__(BLK) k_prolong(LevelArgs A, Tables T, const TC* __restrict__ d,
                                                 TV* __restrict__ U) {
    const int tid = blockIdx.x * BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int g = A.off + lc;
    const int og = g >> 3;
    const TV u = U[g];
    const bool act = TV(tov(__ldg(d + g))) != TV(0);
    const TV ubar = octet_active_mean<TV>(u, act);
    if (valid && act) U[g] = u + (U[__ldg(T.oct_parent + og)] - ubar);
}

// Coarsest level in global memory (one CTA; used when the coarse tail does not fit in
// shared memory): nu sweeps, half red->black then half black->red; fas != 0 completes
// the FAS right-hand side first; prolong != 0 prolongs onto the finer level at the end.
template <class TV, class TC, class TW>
__global__ void __launch_bounds__(1024) k_coarsest(LevelArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                                   TV* __restrict__ B, int nu, int fas, int prolong) {
    const int nb = blockDim.x;
    auto pass = [&](int colour, int mode) {
        for (int base = 0; base < A.ncell; base += nb) {
            const int tid = base + threadIdx.x;
            const bool valid = tid < A.ncell;
            const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
            const int g = A.off + lc;
            const int s = lc & 7;
            const TV u = U[g];
            const TV b = B[g];
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
    if (prolong) {
        for (int c = threadIdx.x; c < A.ncell; c += nb) {
            const int co = T.child_oct[A.off + c];
            if (co >= 0) prolong_children<TV, TC>(C.d, U, co, U[A.off + c]);
        }
    }
}

// ------------------------------------------------------------------ coarse tail
// The smallest levels (levels <= 0: no T faces) run their whole sub-cycle in one CTA
// with every array in shared memory: load, recurse over the tail levels exactly like the
// host driver does (Alg. 4), write back, and optionally prolong the top tail level onto
// the level above it.
struct TailLevel {
    int off;      // first global cell
    int ncell;
    int sbase;    // first cell in the shared arrays
};

struct TailArgs {
    int nlev;                 // L[0] = top (finest) tail level ... L[nlev-1] = coarsest
    TailLevel L[MAXLEV];
    int ncell;                // total cells in the tail
    int mu, nu_pre, nu_post, nu_coarsest;
    int fas, prolong;
};

template <class TV>
struct TailSmem {
    TV *u, *b, *d, *cx, *cy, *cz;
    int* nbr;      // [6][noct_tail] tail-local octet of the same level, -1 wall
    int* par;      // [noct_tail] tail-local parent cell, -1 on the coarsest level
    unsigned char* kids;  // [ncell] 1 if the cell has children
    int noct;
};

template <class TV>
__device__ __forceinline__ TV tail_Au(const TailSmem<TV>& S, int c, int s, TV u, TV dd, const TV cm[3]) {
    const int oc = c >> 3;
    TV Au = dd * u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        const TV ca = cm[a];
        const TV u_in = __shfl_xor_sync(FULL, u, bit);
        const TV ca_in = __shfl_xor_sync(FULL, ca, bit);
        if (s & bit) {
            Au += ca * u_in;
            const int v = S.nbr[(2 * a + 1) * S.noct + oc];
            if (v >= 0) {
                const int ng = 8 * v + (s ^ bit);
                const TV* cc = a == 0 ? S.cx : (a == 1 ? S.cy : S.cz);
                Au += cc[ng] * S.u[ng];
            }
        } else {
            Au += ca_in * u_in;
            const int v = S.nbr[(2 * a) * S.noct + oc];
            if (v >= 0) Au += ca * S.u[8 * v + (s ^ bit)];
        }
    }
    return Au;
}

enum { TP_SWEEP0 = 0, TP_SWEEP1 = 1, TP_FIXB = 2, TP_RESTRICT = 3, TP_PROLONG = 4 };

template <class TV>
__device__ void tail_pass(const TailSmem<TV>& S, const TailLevel& L, int kind, TV scale) {
    for (int base = 0; base < L.ncell; base += blockDim.x) {
        const int tid = base + threadIdx.x;
        const bool valid = tid < L.ncell;
        const int lc = valid ? tid : (L.ncell - 8 + (tid & 7));
        const int c = L.sbase + lc;
        const int s = lc & 7;
        const TV u = S.u[c];
        const TV dd = S.d[c];
        const bool act = dd != TV(0);
        const TV ubar = octet_active_mean<TV>(u, act);
        if (kind == TP_PROLONG) {
            if (valid && act) S.u[c] = u + (S.u[S.par[c >> 3]] - ubar);
            continue;
        }
        const TV cm[3] = {S.cx[c], S.cy[c], S.cz[c]};
        const TV Au = tail_Au<TV>(S, c, s, u, dd, cm);
        const TV b = S.b[c];
        if (kind == TP_FIXB) {
            if (valid && S.kids[c]) S.b[c] = b + Au;
        } else if (kind == TP_RESTRICT) {
            const TV rs = octet_sum<TV>(act ? b - Au : TV(0));
            if (valid && s == 0) {
                const int P = S.par[c >> 3];
                S.b[P] = scale * rs;
                S.u[P] = ubar;
            }
        } else if (valid && act && ((__popc(s) & 1) == kind)) {
            S.u[c] = u + (b - Au) / dd;
        }
    }
    __syncthreads();
}

template <class TV>
__device__ void tail_cycle(const TailSmem<TV>& S, const TailArgs& A, int li, bool fas, TV scale) {
    const TailLevel& L = A.L[li];
    if (fas) tail_pass<TV>(S, L, TP_FIXB, scale);
    if (li == A.nlev - 1) {
        const int half = A.nu_coarsest / 2;
        for (int it = 0; it < half; ++it) { tail_pass<TV>(S, L, 0, scale); tail_pass<TV>(S, L, 1, scale); }
        for (int it = half; it < A.nu_coarsest; ++it) { tail_pass<TV>(S, L, 1, scale); tail_pass<TV>(S, L, 0, scale); }
        return;
    }
    for (int it = 0; it < A.nu_pre; ++it) { tail_pass<TV>(S, L, 0, scale); tail_pass<TV>(S, L, 1, scale); }
    tail_pass<TV>(S, L, TP_RESTRICT, scale);
    for (int k = 0; k < A.mu; ++k) tail_cycle<TV>(S, A, li + 1, k == 0, scale);
    tail_pass<TV>(S, L, TP_PROLONG, scale);
    for (int it = 0; it < A.nu_post; ++it) { tail_pass<TV>(S, L, 1, scale); tail_pass<TV>(S, L, 0, scale); }
}

template <class TV, class TC, class TW>
__global__ void __launch_bounds__(1024) k_tail(TailArgs A, Tables T, Coefs<TC, TW> C, TV* __restrict__ U,
                                               TV* __restrict__ B, TV scale) {
    extern __shared__ __align__(16) unsigned char smem[];
    TailSmem<TV> S;
    const int N = A.ncell, NO = N / 8;
    TV* base = reinterpret_cast<TV*>(smem);
    S.u = base; S.b = base + N; S.d = base + 2 * N; S.cx = base + 3 * N; S.cy = base + 4 * N; S.cz = base + 5 * N;
    S.nbr = reinterpret_cast<int*>(base + 6 * N);
    S.par = S.nbr + 6 * NO;
    S.kids = reinterpret_cast<unsigned char*>(S.par + NO);
    S.noct = NO;
    for (int li = 0; li < A.nlev; ++li) {
        const TailLevel& L = A.L[li];
        for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
            const int g = L.off + c, q = L.sbase + c;
            S.u[q] = U[g];
            S.b[q] = B[g];
            S.d[q] = TV(tov(C.d[g]));
            S.cx[q] = TV(tov(C.cx[g]));
            S.cy[q] = TV(tov(C.cy[g]));
            S.cz[q] = TV(tov(C.cz[g]));
            S.kids[q] = T.child_oct[g] >= 0 ? 1 : 0;
        }
        const int no = L.ncell / 8, ob = L.sbase / 8, og0 = L.off / 8;
        const bool coarsest = li + 1 == A.nlev;
        for (int o = threadIdx.x; o < no; o += blockDim.x) {
            for (int dir = 0; dir < 6; ++dir) {
                const int v = T.nbr[dir * T.noct + og0 + o];
                S.nbr[dir * NO + ob + o] = v >= 0 ? (ob + v) : -1;
            }
            // the parent of an octet of L[li] is a cell of the coarser L[li + 1]
            S.par[ob + o] = coarsest ? -1 : (T.oct_parent[og0 + o] - A.L[li + 1].off + A.L[li + 1].sbase);
        }
    }
    __syncthreads();
    tail_cycle<TV>(S, A, 0, A.fas != 0, scale);
    for (int li = 0; li < A.nlev; ++li) {
        const TailLevel& L = A.L[li];
        for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
            U[L.off + c] = S.u[L.sbase + c];
            B[L.off + c] = S.b[L.sbase + c];
        }
    }
    if (A.prolong) {
        const TailLevel& L = A.L[0];
        for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
            const int co = T.child_oct[L.off + c];
            if (co >= 0) prolong_children<TV, TC>(C.d, U, co, S.u[L.sbase + c]);
        }
    }
}

// Inner values of the outer vector: p_P = mean of P's active children (level m cells
// -> parents at level m-1), used by the composite operator (pbar_P and the coarse side).
template <class TO, class TC>
__global__ void __launch_bounds__(BLK) k_avg(LevelArgs A, Tables T, const TC* __restrict__ d, TO* __restrict__ P) {
    const int tid = blockIdx.x * BLK + threadIdx.x;
    const bool valid = tid < A.ncell;
    const int lc = valid ? tid : (A.ncell - 8 + (tid & 7));
    const int g = A.off + lc;
    const TO u = P[g];
    const bool act = TO(tov(__ldg(d + g))) != TO(0);
    const TO m = octet_active_mean<TO>(u, act);
    if (valid && (lc & 7) == 0) P[__ldg(T.oct_parent + (g >> 3))] = m;
}

// ------------------------------------------------------------------ reductions
// Device scalars of the Krylov loop.
enum {
    S_PAP = 0, S_ALPHA, S_RZ, S_BETA, S_RR, S_RS, S_MEAN, S_BB, S_NS, S_TOL, S_MAXIT, S_K, S_DONE, S_TRUE,
    S_HIST = 16, S_COUNT = 16 + 128
};
enum { OP_NONE = -1, OP_ALPHA = 0, OP_RR = 1, OP_BETA = 2, OP_RZ0 = 3, OP_BB = 4, OP_TRUE = 5 };

// A reduction spread over nb blocks: each block stores its FP64 partial(s) in part[blk]
// (and part[nb + blk]); the last block to arrive sums them in a fixed order and applies
// `op` (the scalar steps of Alg. 1) on the device, then re-arms the counter.
struct Red {
    double* part;
    unsigned* cnt;
    double* S;
    int nb;
    int op;
    double nleaf;
    cudaGraphConditionalHandle cond;
    int set_cond;
};

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

__device__ void red_apply(const Red& R, double sa, double sb) {
    double* S = R.S;
    const bool ns = S[S_NS] != 0.0;
    switch (R.op) {
        case OP_ALPHA: S[S_PAP] = sa; S[S_ALPHA] = sa != 0.0 ? S[S_RZ] / sa : 0.0; break;
        case OP_RZ0: S[S_RZ] = sa; break;
        case OP_BETA: S[S_BETA] = S[S_RZ] != 0.0 ? sa / S[S_RZ] : 0.0; S[S_RZ] = sa; break;
        case OP_BB: {
            const double mean = ns ? sb / R.nleaf : 0.0;
            S[S_MEAN] = mean;
            S[S_BB] = ns ? sa - sb * mean : sa;
            break;
        }
        case OP_RR: {
            const double mean = ns ? sb / R.nleaf : 0.0;
            const double rr = ns ? sa - sb * mean : sa;
            S[S_MEAN] = mean;
            S[S_RR] = rr;
            const int k = (int)S[S_K] + 1;
            S[S_K] = k;
            const double bb = S[S_BB];
            const double rel = bb > 0.0 ? sqrt(fmax(rr, 0.0) / bb) : 0.0;
            if (k < 128) S[S_HIST + k] = rel;
            const bool done = !(rel > S[S_TOL]) || k >= (int)S[S_MAXIT];
            S[S_DONE] = done ? 1.0 : 0.0;
            if (R.set_cond) cudaGraphSetConditional(R.cond, done ? 0u : 1u);
            break;
        }
        case OP_TRUE: {
            const double mean = ns ? sb / R.nleaf : 0.0;
            S[S_TRUE] = ns ? sa - sb * mean : sa;
            break;
        }
        default: break;
    }
}

// Called by every block of a reduction; blk = index of this block within it.
__device__ void red_finish(const Red& R, int blk, double va, double vb, double* sh) {
    __shared__ int last;
    const double ta = block_sum(va, sh);
    const double tb = block_sum(vb, sh);
    if (threadIdx.x == 0) {
        R.part[blk] = ta;
        R.part[R.nb + blk] = tb;
        __threadfence();
        const unsigned prev = atomicAdd(R.cnt, 1u);
        last = prev == (unsigned)(R.nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < R.nb; i += blockDim.x) {
        a += __ldcg(R.part + i);
        b += __ldcg(R.part + R.nb + i);
    }
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    if (threadIdx.x == 0) {
        red_apply(R, sa, sb);
        *R.cnt = 0u;
    }
}

struct MultiLevel {
    int n;
    int off[MAXLEV];
    int ncell[MAXLEV];
    int boff[MAXLEV + 1];   // first block of each level
};

// Composite leaf operator on all tree levels in one launch: Y = A p on leaves, 0 on
// inner cells; (p, A p) over leaves reduced into R (alpha of Alg. 1 when R.op = OP_ALPHA).
template <class TO, class TC, class TW>
__global__ void __launch_bounds__(BLK) k_apply(MultiLevel ML, Tables T, Coefs<TC, TW> C, const TO* __restrict__ P,
                                               TO* __restrict__ Y, Red R) {
    __shared__ double sh[32];
    int l = 0;
    while (l + 1 < ML.n && (int)blockIdx.x >= ML.boff[l + 1]) ++l;
    const int tid = ((int)blockIdx.x - ML.boff[l]) * BLK + threadIdx.x;
    const int ncell = ML.ncell[l], off = ML.off[l];
    const bool valid = tid < ncell;
    const int lc = valid ? tid : (ncell - 8 + (tid & 7));
    const int g = off + lc;
    const int s = lc & 7;
    const TO p = P[g];
    const TO dd = TO(tov(__ldg(C.d + g)));
    const TO cm[3] = {TO(tov(__ldg(C.cx + g))), TO(tov(__ldg(C.cy + g))), TO(tov(__ldg(C.cz + g)))};
    const bool act = dd != TO(0);
    const TO pbar = octet_active_mean<TO>(p, act);
    const TO Ap = stencil_Au<TO, TC, TW>(T, C, P, off, g >> 3, s, p, pbar, dd, cm);
    const bool leaf = __ldg(T.child_oct + g) < 0;
    if (valid) Y[g] = leaf ? Ap : TO(0);
    if (R.op != OP_NONE) {
        const double v = (valid && leaf) ? (double)p * (double)Ap : 0.0;
        red_finish(R, blockIdx.x, v, 0.0, sh);
    }
}

// ----------------------------------------------------------------- PCG vector kernels
template <class TI, class TO>
__global__ void k_scatter(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                          int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[leaf_cell[r]] = TO(in[r]);
}

template <class TI, class TO>
__global__ void k_cast(const TI* __restrict__ in, TO* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = TO(in[i]);
}

template <class TI, class TO>
__global__ void k_gather(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                         int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = TO(in[leaf_cell[r]]);
}

// x += alpha p, r -= alpha Ap over the tree cells (inner cells keep r = 0 since Ap = 0
// there); reduces r.r and sum(r) (OP_RR: convergence test of Alg. 1); optionally b32 = r.
template <class TO, class TB>
__global__ void __launch_bounds__(BLK) k_update(TO* __restrict__ x, TO* __restrict__ r, const TO* __restrict__ p,
                                                const TO* __restrict__ Ap, TB* __restrict__ b32, int n, Red R) {
    __shared__ double sh[32];
    const int i = blockIdx.x * BLK + threadIdx.x;
    const double alpha = R.S[S_ALPHA];
    double rr = 0.0, rs = 0.0;
    if (i < n) {
        x[i] = x[i] + TO(alpha) * p[i];
        const TO rn = r[i] - TO(alpha) * Ap[i];
        r[i] = rn;
        if (b32) b32[i] = TB(rn);
        rr = (double)rn * (double)rn;
        rs = (double)rn;
    }
    red_finish(R, blockIdx.x, rr, rs, sh);
}

// r -= mean on leaves (null-space shift of Sec. 2.2) and b32 = r.
template <class TO, class TB>
__global__ void k_project(TO* __restrict__ r, const uint8_t* __restrict__ flags, const double* __restrict__ S,
                          TB* __restrict__ b32, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    TO v = r[i];
    if (flags[i] & 1) v = v - TO(S[S_MEAN]);
    r[i] = v;
    if (b32) b32[i] = TB(v);
}

// (a, b) and sum(a) over the first n cells, reduced into R
template <class TA, class TB>
__global__ void __launch_bounds__(BLK) k_dot(const TA* __restrict__ a, const TB* __restrict__ b, int n, Red R) {
    __shared__ double sh[32];
    const int i = blockIdx.x * BLK + threadIdx.x;
    double v = 0.0, s = 0.0;
    if (i < n) {
        v = (double)a[i] * (double)b[i];
        s = (double)a[i];
    }
    red_finish(R, blockIdx.x, v, s, sh);
}

// ||b - y||^2 and sum(b - y) over leaves (true residual at exit)
template <class TO>
__global__ void __launch_bounds__(BLK) k_resid(const TO* __restrict__ b, const TO* __restrict__ y,
                                               const uint8_t* __restrict__ flags, int n, Red R) {
    __shared__ double sh[32];
    const int i = blockIdx.x * BLK + threadIdx.x;
    double v = 0.0, s = 0.0;
    if (i < n && (flags[i] & 1)) {
        const double d = (double)b[i] - (double)y[i];
        v = d * d;
        s = d;
    }
    red_finish(R, blockIdx.x, v, s, sh);
}

template <class TO, class TZ>
__global__ void k_pupdate(TO* __restrict__ p, const TZ* __restrict__ z, const double* __restrict__ S, int n,
                          int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = first ? TO(z[i]) : TO(z[i]) + TO(S[S_BETA]) * p[i];
}

// ----------------------------------------------------------------- setup kernels (FP64)

// -beta_f h_f into the face's destination: the - face coefficient of its + cell, or the
// T record weight of a fine leaf's + face.  Flags a negative / non-finite beta.
__global__ void k_face_scatter(const float* __restrict__ beta, const int64_t* __restrict__ slot,
                               const uint8_t* __restrict__ kind, const int32_t* __restrict__ depth,
                               const double* __restrict__ hdepth, int nface, double* __restrict__ cm,
                               double* __restrict__ tw, int* __restrict__ err) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nface) return;
    const float b = beta[f];
    if (!(b >= 0.0f) || !isfinite(b)) atomicOr(err, 1);
    const double w = (double)b * hdepth[depth[f]];
    if (kind[f] == 0) cm[slot[f]] = -w;
    else tw[slot[f]] = -w;
}

struct LevelTab {
    int off[32];
    double h[32];
    int mc;
};

// Per leaf: the - face coefficients the scatter could not write (walls; coarse side of a
// T-junction = (1/2) sum of the fine sub-face weights, Sec. 3.1) and the diagonal = sum of
// the six face weights (Eq. projection-poisson-system).
__global__ void k_leaf_gather(const int32_t* __restrict__ leaf_cell, const int8_t* __restrict__ level,
                              Tables T, LevelTab LT, int4 bc_lo, int2 bc_hi, int nleaf, int ncell,
                              double* __restrict__ dg, double* __restrict__ cm, const double* __restrict__ tw) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nleaf) return;
    const int bc[6] = {bc_lo.x, bc_lo.y, bc_lo.z, bc_lo.w, bc_hi.x, bc_hi.y};
    const int g = leaf_cell[r];
    const int m = level[g];
    const int off = LT.off[m - LT.mc];
    const double h = LT.h[m - LT.mc];
    const int s = (g - off) & 7;
    const int og = g >> 3;
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int bit = 1 << a;
        double* cma = cm + (int64_t)a * ncell;
        // - face
        double wm;
        int nmi = -1;   // same-depth cell on the - side
        bool wall = false;
        if (s & bit) nmi = g ^ bit;
        else {
            const int v = T.nbr[(2 * a) * T.noct + og];
            if (v >= 0) nmi = off + 8 * v + (s ^ bit);
            else if (v == -1) wall = true;
        }
        if (wall) {
            wm = bc[2 * a] ? 2.0 * h : 0.0;
            cma[g] = -wm;
        } else if (nmi >= 0 && T.child_oct[nmi] >= 0) {
            // coarse side: children of nmi with bit a = 1 hold fine + faces in their T record
            const int co = T.child_oct[nmi];
            const int v = T.nbr[(2 * a + 1) * T.noct + co];
            const int t = -2 - v;
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) acc += tw[((2 * a + 1) * 4 + q) * T.nt + t];
            cma[g] = 0.5 * acc;
            wm = -0.5 * acc;
        } else {
            wm = -cma[g];   // regular or fine side of a T-junction (written by the scatter)
        }
        // + face
        double wp;
        int npl = -1;
        wall = false;
        int tplus = -1;
        if (!(s & bit)) npl = g ^ bit;
        else {
            const int v = T.nbr[(2 * a + 1) * T.noct + og];
            if (v >= 0) npl = off + 8 * v + (s ^ bit);
            else if (v == -1) wall = true;
            else tplus = -2 - v;
        }
        if (wall) {
            wp = bc[2 * a + 1] ? 2.0 * h : 0.0;
        } else if (tplus >= 0) {
            wp = -tw[((2 * a + 1) * 4 + sub_index(a, s)) * T.nt + tplus];
        } else if (T.child_oct[npl] >= 0) {
            // coarse side: the four children of npl with bit a = 0 keep the fine - faces
            const int c8 = 8 * T.child_oct[npl];
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
                          int ncell) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= A.ncell / 8) return;
    const int c8 = A.off + 8 * o;
    const int P = T.oct_parent[c8 >> 3];
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
