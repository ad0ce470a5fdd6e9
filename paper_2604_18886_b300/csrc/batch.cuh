// Batched form: many independent octree solves advanced by one launch per phase.
//
// Each problem keeps its own hierarchy (tables, coefficients, vectors, device scalars);
// a launch covers the same step of every problem through a device array of problem
// descriptors and a block map (block -> work item).  Blocks never straddle two problems,
// so per-problem reductions, early exits of converged problems and the warp shuffles of
// the thread-per-cell sweep all stay inside one problem.  Mixed precision only: FP32
// cycle on FP32 coefficients, FP64 Krylov vectors.
#pragma once

#include "octet.cuh"

namespace ocg {

struct BLev {
    int off, ncell, ni;
};

struct BProb {
    Tables T;
    Coefs<float, float> C;
    float* U;             // cycle work vectors, in the cycle layout (cyc)
    float* B;
    double *x, *r, *p, *Ap, *bt, *xt, *yt;
    double* S;            // this problem's Krylov scalars (S_*)
    double* part;         // reduction partials: 3 * max(nbv, nba)
    unsigned* cnt;        // reduction arrival counter
    const uint8_t* flags;
    const float* rem;     // diagonal remainder of the tree cells (outer apply)
    const int32_t* leaf_cell;
    int ntree, nleaf;
    int vb0, nbv;         // vector kernels: first block, blocks
    int ab0, nba;         // composite operator: first block, blocks
    int D, mc;
    int fuse_first;       // the vector kernels that write B form the cycle's first sweep (finest
                          // level swept by launches, not inside the tail): FirstSweep
    BLev L[2 * MAXLEV];   // index m - mc
    TailArgs tail;        // float cycle
};

struct BWork {
    int prob;
    int m;
    int b0;               // first block of this item
    int flags;            // bit 0: prolong onto the finer level / FAS pass; bit 1: fixb
};

struct BRed {
    int op;
    int nprob;
    unsigned* gcnt;                     // problems whose reduction has finished
    cudaGraphConditionalHandle cond;
    int set_cond;
};

__device__ __forceinline__ bool bdone(const BProb& P) { return P.S[S_DONE] != 0.0; }

// Per-problem reduction (the block is block blk of nb of its problem); the last block of
// a problem applies `op` to that problem's scalars (state-changing steps are skipped once
// the problem has converged); with set_cond the last problem to finish sets the WHILE
// condition: continue while any problem has not converged.
template <int NV>
__device__ void bred_finish(const BProb* __restrict__ PP, int pid, int blk, int nb, const BRed& R, double va,
                            double vb, double vc, double* sh) {
    const BProb& P = PP[pid];
    __shared__ int last;
    const double ta = block_sum(va, sh);
    const double tb = block_sum(vb, sh);
    const double tc = NV > 2 ? block_sum(vc, sh) : 0.0;
    if (threadIdx.x == 0) {
        P.part[blk] = ta;
        P.part[nb + blk] = tb;
        if (NV > 2) P.part[2 * nb + blk] = tc;
        __threadfence();
        const unsigned prev = atomicAdd(P.cnt, 1u);
        last = prev == (unsigned)(nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += __ldcg(P.part + i);
        b += __ldcg(P.part + nb + i);
        if (NV > 2) c += __ldcg(P.part + 2 * nb + i);
    }
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    const double sc = NV > 2 ? block_sum(c, sh) : 0.0;
    if (threadIdx.x == 0) {
        const bool frozen = (R.op == OP_ALPHA || R.op == OP_RR || R.op == OP_BETA) && P.S[S_DONE] != 0.0;
        if (!frozen) {
            Red r1{P.part, P.cnt, P.S, nb, R.op, (double)P.nleaf, 0, 0};
            red_apply(r1, sa, sb, sc);
        }
        *P.cnt = 0u;
        if (R.set_cond) {
            __threadfence();
            const unsigned g = atomicAdd(R.gcnt, 1u);
            if (g == (unsigned)(R.nprob - 1)) {
                __threadfence();
                int open = 0;
                for (int q = 0; q < R.nprob; ++q) open |= __ldcg(PP[q].S + S_DONE) == 0.0 ? 1 : 0;
                *R.gcnt = 0u;
                cudaGraphSetConditional(R.cond, open ? 1u : 0u);
            }
        }
    }
}

__device__ __forceinline__ LevelArgs blevel(const BProb& P, int m) {
    const BLev& l = P.L[m - P.mc];
    return LevelArgs{l.off, l.ncell, l.ni};
}

// ------------------------------------------------------------------ cycle phases
// colour sweep / FAS right-hand-side pass of one level of every listed problem, one
// thread per octet
// skip_first: the first colour-0 sweep of a cycle, which the vector kernels already formed
// on the finest level of the problems with fuse_first
__global__ void __launch_bounds__(OBLK) kb_osweep(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                  const int* __restrict__ bmap, int colour, int fixb, int skip_first) {
    const BWork w = W[bmap[blockIdx.x]];
    const BProb& P = PP[w.prob];
    if (bdone(P) || (skip_first && P.fuse_first && w.m == P.D)) return;
    const LevelArgs A = blevel(P, w.m);
    const int o = ((int)blockIdx.x - w.b0) * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    if (fixb) {
        if (w.flags & 2) osweep_octet<float, float, float>(A, P.T, P.C, P.U, P.B, o, 0, 0, 1);
    } else {
        osweep_octet<float, float, float>(A, P.T, P.C, P.U, P.B, o, colour, w.flags & 1, 0);
    }
}

// the same colour sweep, one thread per cell
__global__ void __launch_bounds__(BLK) kb_csweep(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                 const int* __restrict__ bmap, int colour, int skip_first) {
    const BWork w = W[bmap[blockIdx.x]];
    const BProb& P = PP[w.prob];
    if (bdone(P) || (skip_first && P.fuse_first && w.m == P.D)) return;
    const LevelArgs A = blevel(P, w.m);
    csweep_cell<float, float, float>(A, P.T, P.C, P.U, P.B, ((int)blockIdx.x - w.b0) * BLK + threadIdx.x, colour,
                                     w.flags & 1);
}

__global__ void __launch_bounds__(OBLK) kb_orestrict(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                     const int* __restrict__ bmap, float scale) {
    const BWork w = W[bmap[blockIdx.x]];
    const BProb& P = PP[w.prob];
    if (bdone(P)) return;
    const LevelArgs A = blevel(P, w.m);
    const int o = ((int)blockIdx.x - w.b0) * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    orestrict_octet<float, float, float>(A, P.T, P.C, P.U, P.B, scale, o);
}

// the coarse tail of every listed problem, one CTA each (dynamic shared memory sized for
// the largest)
__global__ void __launch_bounds__(512) kb_otail(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                float scale, int fas, int prolong) {
    const BWork w = W[blockIdx.x];
    const BProb& P = PP[w.prob];
    if (bdone(P)) return;
    // a tail that is the problem's finest level (flag 1) is entered from no restriction
    // and prolongs onto no finer level
    const int top = w.flags & 1;
    tail_cycle<float, float, float>(P.tail, top ? 0 : fas, top ? 0 : prolong, P.T, P.C, P.U, P.B, scale);
}

// ------------------------------------------------------------------ Krylov vectors
// Vector kernels: problem = bmap[block], block blk = block - vb0 of nbv, grid-stride over
// the problem's tree cells.
#define BVEC_PROLOGUE                                              \
    const int pid = bmap[blockIdx.x];                              \
    const BProb& P = PP[pid];                                      \
    const int blk = (int)blockIdx.x - P.vb0, nb = P.nbv;           \
    const int i0 = blk * BLK + threadIdx.x, di = nb * BLK;

// U = 0 on the tree cells (the cycle's initial guess) of the problems whose vector kernels
// do not form the first sweep
__global__ void __launch_bounds__(BLK) kb_zero_u(const BProb* __restrict__ PP, const int* __restrict__ bmap) {
    BVEC_PROLOGUE
    if (bdone(P) || P.fuse_first) return;
    for (int i = i0; i < P.ntree; i += di) P.U[cyc(i)] = 0.0f;
}

// B = b on tree cell i and, with fuse_first, the cycle's first sweep in U (FirstSweep)
__device__ __forceinline__ void bput(const BProb& P, int i, float b) {
    P.B[cyc(i)] = b;
    if (P.fuse_first) {
        const BLev& l = P.L[P.D - P.mc];
        const FirstSweep F{P.U, P.C.d, l.off, l.off + l.ncell};
        P.U[cyc(i)] = first_sweep_u(F, i, b);
    }
}

// Per-call input / output of each problem (canonical leaf order).
struct BIO {
    const double* b;
    double* x;
};

// scatter this call's b onto the leaf cells of bt (its inner cells stay 0), zero x and
// p; ||b||^2, sum(b) -> OP_BB
__global__ void __launch_bounds__(BLK) kb_begin(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                const BIO* __restrict__ io, BRed R) {
    __shared__ double sh[32];
    BVEC_PROLOGUE
    for (int i = i0; i < P.ntree; i += di) {
        P.x[i] = 0.0;
        P.p[i] = 0.0;
    }
    const double* bin = io[pid].b;
    double bb = 0.0, bs = 0.0;
    for (int q = i0; q < P.nleaf; q += di) {
        const double v = bin[q];
        P.bt[P.leaf_cell[q]] = v;
        bb += v * v;
        bs += v;
    }
    bred_finish<2>(PP, pid, blk, nb, R, bb, bs, 0.0, sh);
}

// r = bt (after the whole begin scatter), minus the null-space mean; B = r
__global__ void __launch_bounds__(BLK) kb_rinit(const BProb* __restrict__ PP, const int* __restrict__ bmap) {
    BVEC_PROLOGUE
    const double mean = P.S[S_MEAN];
    for (int i = i0; i < P.ntree; i += di) {
        double v = P.bt[i];
        if (P.flags[i] & 1) v -= mean;
        P.r[i] = v;
        bput(P, i, (float)v);
    }
}

// (r, z) with z = U; op OP_RZ0 or OP_BETA
__global__ void __launch_bounds__(BLK) kb_dot_rz(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                 BRed R) {
    __shared__ double sh[32];
    BVEC_PROLOGUE
    double v = 0.0;
    if (!bdone(P))
        for (int i = i0; i < P.ntree; i += di) v += P.r[i] * (double)P.U[cyc(i)];
    bred_finish<2>(PP, pid, blk, nb, R, v, 0.0, 0.0, sh);
}

// p = z (first) or z + beta p
__global__ void __launch_bounds__(BLK) kb_pupdate(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                  int first) {
    BVEC_PROLOGUE
    if (bdone(P)) return;
    const double beta = P.S[S_BETA];
    for (int i = i0; i < P.ntree; i += di) P.p[i] = first ? (double)P.U[cyc(i)] : (double)P.U[cyc(i)] + beta * P.p[i];
}

// x += alpha p, r -= alpha Ap; ||r||^2, sum(r) -> OP_RR (per-problem stop test)
__global__ void __launch_bounds__(BLK) kb_update(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                 BRed R) {
    __shared__ double sh[32];
    BVEC_PROLOGUE
    double rr = 0.0, rs = 0.0;
    if (!bdone(P)) {
        const double alpha = P.S[S_ALPHA];
        const bool ns = P.S[S_NS] != 0.0;
        for (int i = i0; i < P.ntree; i += di) {
            P.x[i] = P.x[i] + alpha * P.p[i];
            const double rn = P.r[i] - alpha * P.Ap[i];
            P.r[i] = rn;
            if (!ns) bput(P, i, (float)rn);
            rr += rn * rn;
            rs += ns ? rn : 0.0;
        }
    }
    bred_finish<2>(PP, pid, blk, nb, R, rr, rs, 0.0, sh);
}

// r -= mean on leaves (null space), B = r; problems without the null space skip
__global__ void __launch_bounds__(BLK) kb_project(const BProb* __restrict__ PP, const int* __restrict__ bmap) {
    BVEC_PROLOGUE
    if (bdone(P) || P.S[S_NS] == 0.0) return;
    const double mean = P.S[S_MEAN];
    for (int i = i0; i < P.ntree; i += di) {
        double v = P.r[i];
        if (P.flags[i] & 1) v -= mean;
        P.r[i] = v;
        bput(P, i, (float)v);
    }
}

// xt = x (FP64 copy for the true residual and the read-out)
__global__ void __launch_bounds__(BLK) kb_copy_x(const BProb* __restrict__ PP, const int* __restrict__ bmap) {
    BVEC_PROLOGUE
    for (int i = i0; i < P.ntree; i += di) P.xt[i] = P.x[i];
}

// ||bt - yt||^2, sum over leaves -> OP_TRUE
__global__ void __launch_bounds__(BLK) kb_resid(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                BRed R) {
    __shared__ double sh[32];
    BVEC_PROLOGUE
    double v = 0.0, s = 0.0;
    for (int i = i0; i < P.ntree; i += di) {
        if (!(P.flags[i] & 1)) continue;
        const double d = P.bt[i] - P.yt[i];
        v += d * d;
        s += d;
    }
    bred_finish<2>(PP, pid, blk, nb, R, v, s, 0.0, sh);
}

// sum of xt over leaves -> OP_XMEAN
__global__ void __launch_bounds__(BLK) kb_xsum(const BProb* __restrict__ PP, const int* __restrict__ bmap, BRed R) {
    __shared__ double sh[32];
    BVEC_PROLOGUE
    double v = 0.0;
    for (int i = i0; i < P.ntree; i += di)
        if (P.flags[i] & 1) v += P.xt[i];
    bred_finish<2>(PP, pid, blk, nb, R, 0.0, v, 0.0, sh);
}

// solution read-out in canonical leaf order (zero mean under the null space)
__global__ void __launch_bounds__(BLK) kb_gather(const BProb* __restrict__ PP, const int* __restrict__ bmap,
                                                 const BIO* __restrict__ io) {
    BVEC_PROLOGUE
    const double mean = P.S[S_NS] != 0.0 ? P.S[S_XMEAN] : 0.0;
    double* xout = io[pid].x;
    for (int q = i0; q < P.nleaf; q += di) xout[q] = P.xt[P.leaf_cell[q]] - mean;
}
#undef BVEC_PROLOGUE

// ------------------------------------------------------------------ composite operator
// child means of one tree level of every listed problem (bottom-up, one launch per level)
__global__ void __launch_bounds__(OBLK) kb_oavg(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                const int* __restrict__ bmap, int which) {
    const BWork w = W[bmap[blockIdx.x]];
    const BProb& P = PP[w.prob];
    if (which == 0 && bdone(P)) return;
    const LevelArgs A = blevel(P, w.m);
    const int o = ((int)blockIdx.x - w.b0) * OBLK + threadIdx.x;
    if (o >= A.ncell / 8) return;
    double* V = which ? P.xt : P.p;
    const int c8 = A.off + 8 * o;
    double v[8];
    float dd[8];
    ld8(V + c8, v);
    ldc8(P.C.d + c8, dd);
    double s = 0.0;
    int n = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (dd[q] != 0.0f) { s += v[q]; ++n; }
    V[__ldg(P.T.oct_parent + (c8 >> 3))] = s * inv_count<double>(n);
}

// Y = A V over all tree levels of every listed problem; which = 0: V = p, Y = Ap, reduces
// (p, Ap) -> alpha; which = 1: V = xt, Y = yt (true residual), no reduction.  Blocks of
// OBLK2 threads, two lanes (z layers) per octet, as the single-problem outer apply.
__global__ void __launch_bounds__(OBLK2) kb_oapply(const BProb* __restrict__ PP, const BWork* __restrict__ W,
                                                   const int* __restrict__ bmap, int which, BRed R) {
    __shared__ double sh[32];
    const BWork w = W[bmap[blockIdx.x]];
    const BProb& P = PP[w.prob];
    const bool skip = which == 0 && bdone(P);
    const LevelArgs A = blevel(P, w.m);
    const int o = ((int)blockIdx.x - w.b0) * OBLK + (threadIdx.x >> 1);
    const double* V = which ? P.xt : P.p;
    double* Y = which ? P.yt : P.Ap;
    DF dot{0.0f, 0.0f}, sum{0.0f, 0.0f};
    if (!skip && o < A.ncell / 8)
        layer_apply_df(P.T, P.C, P.rem, P.flags, VecD{V}, OutD{Y}, A.off, A.ni, o, threadIdx.x & 1,
                       3u << (threadIdx.x & 30), dot, sum);
    if (which == 0) bred_finish<2>(PP, w.prob, (int)blockIdx.x - P.ab0, P.nba, R, df_to_double(dot), 0.0, 0.0, sh);
}

}  // namespace ocg
