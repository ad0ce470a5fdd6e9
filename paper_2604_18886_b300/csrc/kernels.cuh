// libocg device kernels (sm_103a).
//
// Shared helpers, the reductions of the Krylov loop, vector kernels and the FP64 set-up
// kernels (coefficient fill, Alg. 3 coarsening).  The level kernels (operator, sweeps,
// restriction, prolongation) are in octet.cuh.  No tensor cores: the operator is a
// 7-point stencil, bound by memory traffic and latency.  Cell indices fit in int32
// (the host rejects larger trees).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLK = 256;

// Programmatic dependent launch (sm_90 and later): every kernel of this library first waits
// until the grid it depends on has completed and its memory is visible, then lets the next
// grid be scheduled.  Launched with the programmatic-serialization attribute (launch_k),
// the next kernel's blocks are placed on the SMs while this one runs and the gap between
// dependent kernels shrinks; launched without it, the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
constexpr int MAXLEV = 16;

// Storage of the forward cycle's work vectors (u and b of every level).  The cells of an
// octet split into two colours of the red-black sweep, colour(s) = parity of the slot s
// (the octet's first cell has even coordinates): slots 0, 3, 5, 6 and 1, 2, 4, 7, the
// k-th slot of a colour being s = 2k + (parity(k) xor colour), so k = s >> 1.  Each
// aligned group of 8 octets (64 cells) stores the colour-0 cells of its octets first
// (4 per octet, 16 bytes in FP32) and then the colour-1 cells: a colour sweep reads b and
// writes u in whole 32-byte sectors, and reads one 16-byte chunk per neighbouring octet
// (the face neighbours of a colour's cells are all of the other colour).  The map keeps
// every cell inside its group, so it needs only an allocation rounded up to 64 cells
// (cyc_len) starting at cell 0.  The Krylov vectors and the transposed cycle keep the
// plain cell order.
__host__ __device__ __forceinline__ int cyc_colour(int s) { return (0x96 >> s) & 1; }
__host__ __device__ __forceinline__ int cyc(int g) {
    return (g & ~63) | (cyc_colour(g & 7) << 5) | (((g >> 3) & 7) << 2) | ((g & 7) >> 1);
}
// position of the colour-0 chunk of the octet whose first cell is c8 (colour 1: + 32)
__host__ __device__ __forceinline__ int cyc8(int c8) { return (c8 & ~63) | (((c8 >> 3) & 7) << 2); }
__host__ __device__ __forceinline__ int64_t cyc_len(int64_t n) { return (n + 63) & ~(int64_t)63; }
template <bool CY>
__device__ __forceinline__ int vidx(int g) { return CY ? cyc(g) : g; }

struct Tables {
    const int32_t* nbr;        // [6][noct] level-local octet / -1 wall / -2-K T face
    const int32_t* oct_parent; // [noct] global parent cell
    const int32_t* child_oct;  // [ncell] global children octet or -1
    const int32_t* trec;       // [noct] T record of the octet or -1
    int noct;
    int nt;
};

struct LevelArgs {
    int off;      // first global cell of the level
    int ncell;    // multiple of 8
    int ni;       // uniform level: octets per axis (lexicographic octets); 0 = adaptive
};

template <class TC>
struct DiagOf {
    using type = TC;
};
template <>
struct DiagOf<__nv_bfloat16> {
    using type = float;
};

template <class TC, class TW>
struct Coefs {
    // the diagonal is kept in FP32 when the face coefficients are BF16 (conservative
    // diagonal, see k_diag_conservative)
    const typename DiagOf<TC>::type* d;
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

// ------------------------------------------------------------------ reductions
// Device scalars of the Krylov loop.
enum {
    S_PAP = 0, S_ALPHA, S_RZ, S_BETA, S_RR, S_RS, S_MEAN, S_BB, S_NS, S_TOL, S_MAXIT, S_K, S_DONE, S_TRUE,
    S_RHO, S_RHON, S_OMEGA, S_XMEAN, S_APMEAN,
    S_HIST = 24, S_COUNT = 24 + 128
};
enum {
    OP_NONE = -1, OP_ALPHA = 0, OP_RR = 1, OP_BETA = 2, OP_RZ0 = 3, OP_BB = 4, OP_TRUE = 5,
    // BiCGStab (adjoint system) and the zero-mean shift of the returned solution
    OP_BI_INIT = 6, OP_BI_ALPHA = 7, OP_BI_OMEGA = 8, OP_BI_RR = 9, OP_XMEAN = 10
};

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

// Convergence bookkeeping shared by both Krylov loops: iteration count, history, stop
// flag and the WHILE-node condition.
__device__ __forceinline__ void red_converged(const Red& R, double rr) {
    double* S = R.S;
    S[S_RR] = rr;
    const int k = (int)S[S_K] + 1;
    S[S_K] = k;
    const double bb = S[S_BB];
    const double rel = bb > 0.0 ? sqrt(fmax(rr, 0.0) / bb) : 0.0;
    if (k < 128) S[S_HIST + k] = rel;
    const bool done = !(rel > S[S_TOL]) || k >= (int)S[S_MAXIT];
    S[S_DONE] = done ? 1.0 : 0.0;
    if (R.set_cond) cudaGraphSetConditional(R.cond, done ? 0u : 1u);
}

__device__ void red_apply(const Red& R, double sa, double sb, double sc) {
    double* S = R.S;
    const bool ns = S[S_NS] != 0.0;
    switch (R.op) {
        // sb = the sum of A p over the leaves (the pair-stored mixed apply), whose mean the
        // fused update subtracts under the null space
        case OP_ALPHA:
            S[S_PAP] = sa;
            S[S_ALPHA] = sa != 0.0 ? S[S_RZ] / sa : 0.0;
            S[S_APMEAN] = ns ? sb / R.nleaf : 0.0;
            break;
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
            S[S_MEAN] = mean;
            red_converged(R, ns ? sa - sb * mean : sa);
            break;
        }
        case OP_TRUE: {
            const double mean = ns ? sb / R.nleaf : 0.0;
            S[S_TRUE] = ns ? sa - sb * mean : sa;
            break;
        }
        // BiCGStab: sa = (rhat, r) with rhat = r = b after the null-space shift
        case OP_BI_INIT: {
            S[S_RHON] = sa;
            S[S_RHO] = S[S_ALPHA] = S[S_OMEGA] = 1.0;
            S[S_BETA] = sa;
            S[S_K] = 0.0;
            const double bb = S[S_BB];
            const bool done = !(bb > 0.0) || !(sqrt(fmax(sa, 0.0) / bb) > S[S_TOL]) || (int)S[S_MAXIT] <= 0;
            S[S_DONE] = done ? 1.0 : 0.0;
            if (R.set_cond) cudaGraphSetConditional(R.cond, done ? 0u : 1u);
            break;
        }
        case OP_BI_ALPHA: S[S_ALPHA] = sa != 0.0 ? S[S_RHON] / sa : 0.0; break;   // sa = (rhat, v)
        case OP_BI_OMEGA: S[S_OMEGA] = sb != 0.0 ? sa / sb : 0.0; break;          // (t, s) / (t, t)
        case OP_BI_RR: {
            // sa = ||r||^2, sb = sum(r), sc = (rhat, r); rhat has zero mean under the
            // null space, so the shift r -= mean leaves (rhat, r) unchanged
            const double mean = ns ? sb / R.nleaf : 0.0;
            S[S_MEAN] = mean;
            red_converged(R, ns ? sa - sb * mean : sa);
            S[S_RHO] = S[S_RHON];
            S[S_RHON] = sc;
            const double den = S[S_RHO] * S[S_OMEGA];
            S[S_BETA] = den != 0.0 ? (sc * S[S_ALPHA]) / den : 0.0;
            break;
        }
        case OP_XMEAN: S[S_XMEAN] = ns ? sb / R.nleaf : 0.0; break;
        default: break;
    }
}

// Called by every block of a reduction; blk = index of this block within it.  NV = 2 or
// 3 partial sums per block (part holds NV * nb doubles).
template <int NV = 2>
__device__ void red_finish(const Red& R, int blk, double va, double vb, double vc, double* sh) {
    __shared__ int last;
    const double ta = block_sum(va, sh);
    const double tb = block_sum(vb, sh);
    const double tc = NV > 2 ? block_sum(vc, sh) : 0.0;
    if (threadIdx.x == 0) {
        R.part[blk] = ta;
        R.part[R.nb + blk] = tb;
        if (NV > 2) R.part[2 * R.nb + blk] = tc;
        __threadfence();
        const unsigned prev = atomicAdd(R.cnt, 1u);
        last = prev == (unsigned)(R.nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < R.nb; i += blockDim.x) {
        a += __ldcg(R.part + i);
        b += __ldcg(R.part + R.nb + i);
        if (NV > 2) c += __ldcg(R.part + 2 * R.nb + i);
    }
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    const double sc = NV > 2 ? block_sum(c, sh) : 0.0;
    if (threadIdx.x == 0) {
        red_apply(R, sa, sb, sc);
        *R.cnt = 0u;
    }
}
__device__ __forceinline__ void red_finish(const Red& R, int blk, double va, double vb, double* sh) {
    red_finish<2>(R, blk, va, vb, 0.0, sh);
}

// ----------------------------------------------------------------- pair-of-FP32 arithmetic
// B300 executes FP64 instructions, conversions between FP32 and FP64 included, at 1/64 of
// the FP32 rate.  These helpers convert exactly with integer operations and evaluate
// sums and products of binary64 values as pairs of binary32 (hi, lo) with error-free
// transformations (TwoSum, TwoProd by FMA; T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971).
struct DF {
    float hi, lo;   // value hi + lo; lo is not kept normalised inside a computation
};
// TwoSum (Knuth): s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// a += x, the rounding error of the leading parts carried into lo
__device__ __forceinline__ void df_acc(DF& a, DF x) {
    float s, e;
    two_sum(a.hi, x.hi, s, e);
    a.hi = s;
    a.lo = a.lo + (e + x.lo);
}
// a += c exactly up to the rounding of lo (accumulation of FP32 coefficients)
__device__ __forceinline__ void df_acc_f(DF& a, float c) {
    float s, e;
    two_sum(a.hi, c, s, e);
    a.hi = s;
    a.lo = a.lo + e;
}
__device__ __forceinline__ DF df_diff(DF x, DF y) {
    float s, e;
    two_sum(x.hi, -y.hi, s, e);
    return {s, e + (x.lo - y.lo)};
}
// x * c with the product of the leading parts exact (FMA)
__device__ __forceinline__ DF df_scale(DF x, float c) {
    const float p = x.hi * c;
    return {p, fmaf(x.lo, c, fmaf(x.hi, c, -p))};
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = x.hi * y.hi;
    return {p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)))};
}
__device__ __forceinline__ DF df_norm(DF x) {
    const float s = x.hi + x.lo;
    return {s, x.lo - (s - x.hi)};
}
// s / n for a count 0 <= n <= 8 (the mean of n active cells; 0 for n = 0).  Scaling by
// 1/n is exact for n = 1, 2, 4, 8; otherwise hi = s.hi (1/n) is within two ulps of the
// quotient, so the remainder s.hi - n hi is exact in one FMA, and lo = (remainder + s.lo)/n
// carries the rest to about 2^-47 of the mean.
__device__ __forceinline__ DF df_div_count(DF s, int n) {
    if (n == 0) return DF{0.0f, 0.0f};
    if ((n & (n - 1)) == 0) {
        const float ic = n == 8 ? 0.125f : (n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.0f));
        return DF{s.hi * ic, s.lo * ic};
    }
    const float ic = 1.0f / (float)n;
    const float hi = s.hi * ic;
    const float rem = fmaf(-hi, (float)n, s.hi);
    const float lo = (rem + s.lo) * ic;
    const float t = hi + lo;
    return DF{t, lo - (t - hi)};
}

// binary64 -> (hi, lo): hi = sign, exponent and leading 23 fraction bits (truncated), lo =
// the remaining 29 fraction bits rounded to 24; integer operations only.  |v| < 2^-126 is
// flushed to 0, |v| >= 2^128 becomes an infinity or NaN in hi; lo is dropped when |v| <
// 2^-74 (then the pair keeps 24 bits).
__device__ __forceinline__ DF df_split(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned h32 = (unsigned)(b >> 32);
    const unsigned sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7FFu);   // biased binary64 exponent
    const unsigned hib = sign | ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    const float lo = __uint2float_rn((unsigned)b & 0x1FFFFFFFu) * __uint_as_float((unsigned)(e - 948) << 23);
    const bool normal = (e >= 897) & (e <= 1150);
    const unsigned big = sign | 0x7F800000u | ((b & 0xFFFFFFFFFFFFFull) ? 0x400000u : 0u);
    const float hi = __uint_as_float(normal ? hib : (e < 897 ? sign : big));
    return {hi, (normal & (e >= 949)) ? __uint_as_float(__float_as_uint(lo) | sign) : 0.0f};
}
// binary32 -> binary64 by bits (exact; subnormal floats are flushed to 0)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (ex == 0u) return __longlong_as_double((long long)sign);
    const unsigned long long e64 = ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex - 127u + 1023u);
    return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double df_to_double(DF x) {
    const DF n = df_norm(x);
    return f2d_bits(n.hi) + f2d_bits(n.lo);
}

// FP64 -> FP32 rounded to nearest (through the pair: hi + lo in one FP32 addition)
__device__ __forceinline__ float d2f_bits(double v) {
    const DF p = df_split(v);
    return p.hi + p.lo;
}
template <class TO, class TI>
__device__ __forceinline__ TO cvt(TI v) { return TO(v); }
template <>
__device__ __forceinline__ double cvt<double, float>(float v) { return f2d_bits(v); }
template <>
__device__ __forceinline__ float cvt<float, double>(double v) { return d2f_bits(v); }

// ----------------------------------------------------------------- PCG vector kernels
// CY: out in the cycle layout (cyc)
template <class TI, class TO, bool CY = false>
__global__ void k_scatter(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                          int n) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[vidx<CY>(leaf_cell[r])] = TO(in[r]);
}

template <class TI, class TO>
__global__ void k_cast(const TI* __restrict__ in, TO* __restrict__ out, int n) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = TO(in[i]);
}

// r -= a over the tree cells (the warm start's r = b - A x0)
template <class T>
__global__ void k_sub(T* __restrict__ r, const T* __restrict__ a, int n) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = r[i] - a[i];
}

// CY: in in the cycle layout (cyc)
template <class TI, class TO, bool CY = false>
__global__ void k_gather(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                         int n) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = TO(in[vidx<CY>(leaf_cell[r])]);
}

// The first step of the next preconditioner application, fused into the kernel that writes
// the cycle's right-hand side b32 (F.u32 set, FP32 cycles): the cycle starts from u = 0, so
// its first step, the colour-0 sweep of the finest level, sets u = b / c on that level's
// active colour-0 cells (every neighbour and T ghost is 0) and leaves the other cells at 0.
// The kernel then writes that u over the tree cells (cycle layout) beside b32, in the
// sweep's arithmetic (b rounded to FP32, then the same FP32 division), and the cycle skips
// both the zeroing of u and that sweep.  [d0, d1) are the finest level's cells, d its FP32
// diagonal in cell order.
struct FirstSweep {
    float* u32;
    const float* d;
    int d0, d1;
};
__device__ __forceinline__ float first_sweep_u(const FirstSweep& F, int i, float b) {
    if (i < F.d0 || i >= F.d1 || cyc_colour(i & 7) != 0) return 0.0f;
    const float c = F.d[i];
    return c != 0.0f ? __fdividef(b, c) : 0.0f;
}
__device__ __forceinline__ void first_sweep_store(const FirstSweep& F, int i, float b) {
    if (F.u32) F.u32[cyc(i)] = first_sweep_u(F, i, b);
}
__device__ __forceinline__ void first_sweep_store(const FirstSweep&, int, double) {}
// x += alpha p, r -= alpha Ap over the tree cells (inner cells keep r = 0 since Ap = 0
// there); reduces r.r and sum(r) (OP_RR: convergence test of Alg. 1); optionally b32 = r
// (b32 in the cycle layout when CY).
template <class TO, class TB, bool SUM, bool CY = false>
__global__ void __launch_bounds__(BLK) k_update(TO* __restrict__ x, TO* __restrict__ r, const TO* __restrict__ p,
                                                const TO* __restrict__ Ap, TB* __restrict__ b32, int n, Red R,
                                                FirstSweep F) {
    pdl_enter();
    __shared__ double sh[32];
    const TO alpha = TO(R.S[S_ALPHA]);
    double rr = 0.0, rs = 0.0;
    const int st = gridDim.x * BLK;
    int i = blockIdx.x * BLK + threadIdx.x;
    // four independent elements per thread and pass keep enough loads in flight
    for (; i + 3 * st < n; i += 4 * st) {
        TO xv[4], pv[4], rv[4], av[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { xv[q] = x[i + q * st]; pv[q] = p[i + q * st]; rv[q] = r[i + q * st]; av[q] = Ap[i + q * st]; }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[i + q * st] = xv[q] + alpha * pv[q];
            const TO rn = rv[q] - alpha * av[q];
            r[i + q * st] = rn;
            if (b32) {
                const TB bv = cvt<TB>(rn);
                b32[vidx<CY>(i + q * st)] = bv;
                first_sweep_store(F, i + q * st, bv);
            }
            const double rd = (double)rn;
            rr += rd * rd;
            if (SUM) rs += rd;
        }
    }
    for (; i < n; i += st) {
        x[i] = x[i] + alpha * p[i];
        const TO rn = r[i] - alpha * Ap[i];
        r[i] = rn;
        if (b32) {
            const TB bv = cvt<TB>(rn);
            b32[vidx<CY>(i)] = bv;
            first_sweep_store(F, i, bv);
        }
        const double rd = (double)rn;
        rr += rd * rd;
        if (SUM) rs += rd;
    }
    red_finish(R, blockIdx.x, rr, rs, sh);
}

// The update of k_update for the mixed PCG, whose p is kept as FP32 pairs (hi, lo) that
// the outer apply reads without conversion: x += alpha p (p = hi + lo exactly in
// binary64), r -= alpha A p, b32 = r, ||r||^2; four elements per thread and pass.  Under
// the null space (NS) the zero-mean shift of r (Sec. 2.2) is fused in: r had zero mean, so
// r - alpha (A p - mean(A p)) on the leaves is the shifted residual, the mean of A p
// coming from the apply's reduction (S_APMEAN).  b32 is the forward cycle's b (cycle
// layout).
template <bool NS>
__global__ void __launch_bounds__(BLK) k_update_pp(double* __restrict__ x, double* __restrict__ r,
                                                   const float* __restrict__ phi, const float* __restrict__ plo,
                                                   const double* __restrict__ Ap, const uint8_t* __restrict__ flags,
                                                   float* __restrict__ b32, int n, Red R, FirstSweep F) {
    pdl_enter();
    __shared__ double sh[32];
    const double alpha = R.S[S_ALPHA];
    const double shift = NS ? alpha * R.S[S_APMEAN] : 0.0;
    double rr = 0.0;
    const int st = gridDim.x * BLK;
    int i = blockIdx.x * BLK + threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {
        double xv[4], rv[4], av[4];
        float hv[4], lv[4];
        uint8_t fv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xv[q] = x[i + q * st]; rv[q] = r[i + q * st]; av[q] = Ap[i + q * st];
            hv[q] = phi[i + q * st]; lv[q] = plo[i + q * st];
            fv[q] = NS ? flags[i + q * st] : 0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[i + q * st] = xv[q] + alpha * (f2d_bits(hv[q]) + f2d_bits(lv[q]));
            double rn = rv[q] - alpha * av[q];
            if (NS && (fv[q] & 1)) rn = rn + shift;
            r[i + q * st] = rn;
            const float bf = d2f_bits(rn);
            b32[cyc(i + q * st)] = bf;
            if (F.u32) F.u32[cyc(i + q * st)] = first_sweep_u(F, i + q * st, bf);
            rr += rn * rn;
        }
    }
    for (; i < n; i += st) {
        x[i] = x[i] + alpha * (f2d_bits(phi[i]) + f2d_bits(plo[i]));
        double rn = r[i] - alpha * Ap[i];
        if (NS && (flags[i] & 1)) rn = rn + shift;
        r[i] = rn;
        const float bf = d2f_bits(rn);
        b32[cyc(i)] = bf;
        if (F.u32) F.u32[cyc(i)] = first_sweep_u(F, i, bf);
        rr += rn * rn;
    }
    red_finish(R, blockIdx.x, rr, 0.0, sh);
}

// p = z + beta p (first: p = z) for p kept as FP32 pairs, in pair arithmetic (beta split
// once, TwoProd by FMA, TwoSum; about 2^-47 relative, no FP64 instruction): the same p
// then enters both x += alpha p and the apply, so CG's recurrences stay consistent.  z is
// the forward cycle's u (cycle layout).
template <class TZ>
__global__ void k_pupdate_pp(float* __restrict__ hi, float* __restrict__ lo, const TZ* __restrict__ z,
                             const double* __restrict__ S, int n, int first) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float zi = (float)z[cyc(i)];
    DF v{zi, 0.0f};
    if (!first) {
        v = df_mul(df_split(S[S_BETA]), DF{hi[i], lo[i]});
        df_acc_f(v, zi);
        v = df_norm(v);
    }
    hi[i] = v.hi;
    lo[i] = v.lo;
}

// r -= mean on leaves (null-space shift of Sec. 2.2) and b32 = r (cycle layout when CY).
template <class TO, class TB, bool CY = false>
__global__ void k_project(TO* __restrict__ r, const uint8_t* __restrict__ flags, const double* __restrict__ S,
                          TB* __restrict__ b32, int n, FirstSweep F) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    TO v = r[i];
    if (flags[i] & 1) v = v - TO(S[S_MEAN]);
    r[i] = v;
    if (b32) {
        const TB bv = cvt<TB>(v);
        b32[vidx<CY>(i)] = bv;
        first_sweep_store(F, i, bv);
    }
}

// (a, b) and sum(a) over the first n cells, reduced into R
// (a, b) over the first n cells; with SUM also sum(a) (the null-space mean of Sec. 2.2);
// CY: b in the cycle layout
template <class TA, class TB, bool SUM, bool CY = false>
__global__ void __launch_bounds__(BLK) k_dot(const TA* __restrict__ a, const TB* __restrict__ b, int n, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    double v = 0.0, s = 0.0;
    const int st = gridDim.x * BLK;
    int i = blockIdx.x * BLK + threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {
        TA av[4];
        TB bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { av[q] = a[i + q * st]; bv[q] = b[vidx<CY>(i + q * st)]; }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double ai = cvt<double>(av[q]);
            v += ai * cvt<double>(bv[q]);
            if (SUM) s += ai;
        }
    }
    for (; i < n; i += st) {
        const double ai = cvt<double>(a[i]);
        v += ai * cvt<double>(b[vidx<CY>(i)]);
        if (SUM) s += ai;
    }
    red_finish(R, blockIdx.x, v, s, sh);
}

// ||b - y||^2 and sum(b - y) over leaves (true residual at exit)
template <class TO>
__global__ void __launch_bounds__(BLK) k_resid(const TO* __restrict__ b, const TO* __restrict__ y,
                                               const uint8_t* __restrict__ flags, int n, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    double v = 0.0, s = 0.0;
    for (int i = blockIdx.x * BLK + threadIdx.x; i < n; i += gridDim.x * BLK) {
        if (!(flags[i] & 1)) continue;
        const double d = (double)b[i] - (double)y[i];
        v += d * d;
        s += d;
    }
    red_finish(R, blockIdx.x, v, s, sh);
}

// Solution read-out: out[rank] = in[cell] - S[S_XMEAN] (zero mean under the null space).
template <class TI, class TO>
__global__ void k_gather_shift(const TI* __restrict__ in, TO* __restrict__ out, const int32_t* __restrict__ leaf_cell,
                               const double* __restrict__ S, int n) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = TO((double)in[leaf_cell[r]] - S[S_XMEAN]);
}

// ------------------------------------------------------- BiCGStab (adjoint system)
// Right-preconditioned BiCGStab (van der Vorst 1992) over the tree cells; the scalars
// alpha, beta, omega, rho live in S and are formed by the reductions (OP_BI_*).
// p = r + beta (p - omega v); b32 = p (the cycle's right-hand side)
template <class TO, class TB>
__global__ void k_bi_p(TO* __restrict__ p, const TO* __restrict__ r, const TO* __restrict__ v,
                       TB* __restrict__ b32, const double* __restrict__ S, int n) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TO pn = r[i] + TO(S[S_BETA]) * (p[i] - TO(S[S_OMEGA]) * v[i]);
    p[i] = pn;
    b32[i] = TB(pn);
}

// s = r - alpha v; b32 = s
template <class TO, class TB>
__global__ void k_bi_s(TO* __restrict__ s, const TO* __restrict__ r, const TO* __restrict__ v,
                       TB* __restrict__ b32, const double* __restrict__ S, int n) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TO sn = r[i] - TO(S[S_ALPHA]) * v[i];
    s[i] = sn;
    b32[i] = TB(sn);
}

// (t, s) and (t, t)
template <class TO>
__global__ void __launch_bounds__(BLK) k_dot2(const TO* __restrict__ t, const TO* __restrict__ s, int n, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    double ts = 0.0, tt = 0.0;
    for (int i = blockIdx.x * BLK + threadIdx.x; i < n; i += gridDim.x * BLK) {
        const double ti = (double)t[i];
        ts += ti * (double)s[i];
        tt += ti * ti;
    }
    red_finish(R, blockIdx.x, ts, tt, sh);
}

// x += alpha ph + omega sh; r = s - omega t; reduces ||r||^2, sum(r), (rhat, r)
template <class TO>
__global__ void __launch_bounds__(BLK) k_bi_x(TO* __restrict__ x, TO* __restrict__ r, const TO* __restrict__ s,
                                              const TO* __restrict__ t, const TO* __restrict__ ph,
                                              const TO* __restrict__ shv, const TO* __restrict__ rhat, int n, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    const TO alpha = TO(R.S[S_ALPHA]), omega = TO(R.S[S_OMEGA]);
    double rr = 0.0, rs = 0.0, rh = 0.0;
    for (int i = blockIdx.x * BLK + threadIdx.x; i < n; i += gridDim.x * BLK) {
        x[i] = x[i] + alpha * ph[i] + omega * shv[i];
        const TO rn = s[i] - omega * t[i];
        r[i] = rn;
        const double rd = (double)rn;
        rr += rd * rd;
        rs += rd;
        rh += (double)rhat[i] * rd;
    }
    red_finish<3>(R, blockIdx.x, rr, rs, rh, sh);
}

// ------------------------------------------------------------------ adjoint kernels
// dL/dbeta_f = -lambda^T (dA/dbeta_f) p per canonical face: -h (l_a - l_b)(p_a - p_b) for a
// face between equal-depth leaves a (- side) and b, -(h/2)(l_i - l_K)(pbar_P - p_K) for a T
// sub-face of the fine leaf i against the coarser leaf K, P = parent of i, whose entry of P
// holds the mean of its children.  The fine side of a T face is the - leaf for kind 1
// (T-record faces) and the + leaf when the - leaf is shallower than the face.
struct FaceHs {
    double h[32];   // face size per depth
};
__global__ void k_face_grad(int nface, const int32_t* __restrict__ fminus, const int32_t* __restrict__ fplus,
                            const uint8_t* __restrict__ fkind, const int8_t* __restrict__ fdepth,
                            const int32_t* __restrict__ leaf_cell, const int8_t* __restrict__ level,
                            const int32_t* __restrict__ oct_parent, FaceHs H, const double* __restrict__ P,
                            const double* __restrict__ Lm, double* __restrict__ out) {
    pdl_enter();
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nface) return;
    const int ga = leaf_cell[fminus[f]], gb = leaf_cell[fplus[f]];
    const int d = fdepth[f];
    const double h = H.h[d];
    if (fkind[f] == 0 && level[ga] == d) {
        out[f] = -h * (Lm[ga] - Lm[gb]) * (P[ga] - P[gb]);
        return;
    }
    const int gi = fkind[f] == 1 ? ga : gb, gK = fkind[f] == 1 ? gb : ga;
    const int par = oct_parent[gi >> 3];
    out[f] = -0.5 * h * (Lm[gi] - Lm[gK]) * (P[par] - P[gK]);
}

// sum of x over the leaves (flags bit 0), into the second slot of R
__global__ void __launch_bounds__(BLK) k_leafsum(const double* __restrict__ x, const uint8_t* __restrict__ flags,
                                                 int n, Red R) {
    pdl_enter();
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = blockIdx.x * BLK + threadIdx.x; i < n; i += gridDim.x * BLK)
        if (flags[i] & 1) v += x[i];
    red_finish(R, blockIdx.x, 0.0, v, sh);
}

// p = z (first) or z + beta p; CY: z in the cycle layout
template <class TO, class TZ, bool CY = false>
__global__ void k_pupdate(TO* __restrict__ p, const TZ* __restrict__ z, const double* __restrict__ S, int n,
                          int first) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TO zi = cvt<TO>(z[vidx<CY>(i)]);
    p[i] = first ? zi : zi + TO(S[S_BETA]) * p[i];
}

// ----------------------------------------------------------------- setup kernels (FP64)

// Geometric coarsening (ablation): cells idx[q] take d[q] (only where Alg. 3 gave a nonzero
// diagonal, i.e. the cell has active children) and the - face coefficients cx, cy, cz.
__global__ void k_set_coefs(int n, const int64_t* __restrict__ idx, const double* __restrict__ d,
                            const double* __restrict__ cx, const double* __restrict__ cy,
                            const double* __restrict__ cz, double* __restrict__ D, double* __restrict__ CX,
                            double* __restrict__ CY, double* __restrict__ CZ) {
    pdl_enter();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t g = idx[q];
    if (D[g] != 0.0) D[g] = d[q];
    CX[g] = cx[q];
    CY[g] = cy[q];
    CZ[g] = cz[q];
}


// -beta_f h_f into the face's destination: the - face coefficient of its + cell, or the
// T record weight of a fine leaf's + face.  Flags a negative / non-finite beta.
__global__ void k_face_scatter(const float* __restrict__ beta, const int64_t* __restrict__ slot,
                               const uint8_t* __restrict__ kind, const int8_t* __restrict__ depth,
                               const double* __restrict__ hdepth, int nface, double* __restrict__ cm,
                               double* __restrict__ tw, int* __restrict__ err) {
    pdl_enter();
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
    pdl_enter();
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
            const int t = T.trec[co];
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
            else tplus = T.trec[og];
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
    pdl_enter();
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
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

template <>
__global__ void k_convert<__nv_bfloat16>(const double* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn((float)in[i]);
}

}  // namespace ocg
