// libocg: C ABI, hierarchy set-up, the mu-cycle driver and the PCG loop.
// Every arithmetic step of the solve runs in the kernels of kernels.cuh; this file only
// allocates device memory, uploads the octree tables and sequences launches on the
// caller's stream.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ocg.h"
#include "kernels.cuh"
#include "octree_host.h"

using namespace ocg;

namespace {

thread_local std::string g_err;

struct Status : std::runtime_error {
    int code;
    Status(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) throw Status(OCG_ENOMEM, std::string(what) + ": out of device memory");
        throw Status(OCG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void ck_launch(const char* what) { ck(cudaGetLastError(), what); }

template <class T>
T* dalloc(int64_t n) {
    void* p = nullptr;
    if (n <= 0) n = 1;
    ck(cudaMalloc(&p, (size_t)n * sizeof(T)), "cudaMalloc");
    return (T*)p;
}

template <class T>
T* dupload(const std::vector<T>& v) {
    T* p = dalloc<T>((int64_t)v.size());
    if (!v.empty()) ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
    return p;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

template <class F>
int guard(F&& f) {
    try {
        f();
        return OCG_OK;
    } catch (const Status& s) {
        g_err = s.what();
        return s.code;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return OCG_ENOMEM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return OCG_EINVAL;
    }
}

inline unsigned nblk(int64_t n, int b = BLK) { return (unsigned)((n + b - 1) / b); }

std::atomic<int64_t> g_launches{0};

struct Probe {
    int kind = OCG_PROBE_OFF;
    int level = 0;
    std::vector<cudaEvent_t> ev;   // pairs
    int64_t used = 0;              // events used so far
    int64_t cells = 0;
    ~Probe() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    bool on(int k, int m) const { return kind == k && level == m; }
    void begin(cudaStream_t st) {
        if (used + 2 > (int64_t)ev.size()) {
            for (int q = 0; q < 64; ++q) {
                cudaEvent_t e;
                ck(cudaEventCreate(&e), "cudaEventCreate");
                ev.push_back(e);
            }
        }
        ck(cudaEventRecord(ev[used], st), "cudaEventRecord");
    }
    void end(cudaStream_t st) {
        ck(cudaEventRecord(ev[used + 1], st), "cudaEventRecord");
        used += 2;
    }
};

// Launch wrapper: counts launches and brackets the probed kernel with events.
template <class F>
void launch(Probe* pr, int kind, int m, int64_t cells, cudaStream_t st, F&& f) {
    const bool p = pr && pr->on(kind, m);
    if (p) {
        pr->cells = cells;
        pr->begin(st);
    }
    f();
    ++g_launches;
    if (p) pr->end(st);
}

}  // namespace

struct ocg_octree {
    HostTree H;
    // device copies of the tables, uploaded by the first hierarchy set-up
    mutable bool on_device = false;
    mutable int32_t *nbr = nullptr, *oct_parent = nullptr, *child_oct = nullptr, *tK = nullptr,
                    *leaf_cell = nullptr;
    mutable uint8_t* flags = nullptr;
    mutable int8_t* level = nullptr;
    mutable int64_t* fslot = nullptr;
    mutable uint8_t* fkind = nullptr;
    mutable int32_t* fdepth = nullptr;

    void upload() const {
        if (on_device) return;
        nbr = dupload(H.nbr);
        oct_parent = dupload(H.oct_parent);
        child_oct = dupload(H.child_oct);
        tK = dupload(H.tK);
        leaf_cell = dupload(H.leaf_cell);
        flags = dupload(H.cell_flags);
        level = dupload(H.cell_level);
        fslot = dupload(H.f_slot);
        fkind = dupload(H.f_kind);
        fdepth = dupload(H.f_depth);
        on_device = true;
    }

    Tables tables() const { return Tables{nbr, oct_parent, child_oct, tK, H.noct, H.nt}; }
    LevelArgs largs(int m) const { return LevelArgs{H.L(m).off, H.L(m).ncell}; }
    ~ocg_octree() {
        dfree(nbr); dfree(oct_parent); dfree(child_oct); dfree(tK); dfree(leaf_cell);
        dfree(flags); dfree(level); dfree(fslot); dfree(fkind); dfree(fdepth);
    }
};

struct ocg_hier {
    const ocg_octree* t = nullptr;
    ocg_mg_params prm{};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    bool ns_auto = false;
    double* c64[4] = {nullptr, nullptr, nullptr, nullptr};
    double* tw64 = nullptr;
    float* c32[4] = {nullptr, nullptr, nullptr, nullptr};
    float* tw32 = nullptr;
    __nv_bfloat16* c16[4] = {nullptr, nullptr, nullptr, nullptr};
    // work space
    double* S = nullptr;       // device scalars
    double* hS = nullptr;      // pinned host mirror
    double* part = nullptr;    // block partials
    int64_t npart = 0;
    void* vec[8] = {};         // x, r, p, Ap (outer type), U, B (cycle type), xt, yt
    size_t vec_bytes[8] = {};
    Probe probe;

    Coefs<double, double> C64() const { return {c64[0], c64[1], c64[2], c64[3], tw64}; }
    Coefs<float, float> C32() const { return {c32[0], c32[1], c32[2], c32[3], tw32}; }
    Coefs<__nv_bfloat16, float> C16() const { return {c16[0], c16[1], c16[2], c16[3], tw32}; }

    void* vec_of(int i, size_t bytes) {
        if (vec_bytes[i] < bytes) {
            dfree(vec[i]);
            vec[i] = nullptr;
            vec_bytes[i] = 0;
            ck(cudaMalloc(&vec[i], bytes), "cudaMalloc work vector");
            vec_bytes[i] = bytes;
        }
        return vec[i];
    }
    ~ocg_hier() {
        for (int i = 0; i < 4; ++i) { dfree(c64[i]); dfree(c32[i]); dfree(c16[i]); }
        dfree(tw64); dfree(tw32); dfree(S); dfree(part);
        if (hS) cudaFreeHost(hS);
        for (auto& v : vec) dfree(v);
    }
};

namespace {

// ------------------------------------------------------------------ mu-cycle driver
template <class TV>
struct Cycle {
    ocg_hier* h;
    TV* U;
    TV* B;
    cudaStream_t st;

    const HostTree& H() const { return h->t->H; }

    template <class F>
    void with_coefs(int m, F&& f) {
        if constexpr (std::is_same<TV, double>::value) {
            f(h->C64());
        } else {
            if (h->prm.bf16_coarse && m < H().D) f(h->C16());
            else f(h->C32());
        }
    }
    void fixb(int m) {
        with_coefs(m, [&](auto C) {
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
            const LevelArgs A = h->t->largs(m);
            launch(&h->probe, -1, m, A.ncell, st, [&] {
                k_sweep<TV, TC, TW, MODE_FIXB><<<nblk(A.ncell), BLK, 0, st>>>(A, h->t->tables(), C, U, B, 0);
            });
        });
        ck_launch("fixb");
    }
    void sweep(int m, int colour) {
        with_coefs(m, [&](auto C) {
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
            const LevelArgs A = h->t->largs(m);
            launch(&h->probe, OCG_PROBE_SWEEP, m, A.ncell, st, [&] {
                k_sweep<TV, TC, TW, MODE_SWEEP><<<nblk(A.ncell), BLK, 0, st>>>(A, h->t->tables(), C, U, B, colour);
            });
        });
        ck_launch("sweep");
    }
    void restrict_(int m) {
        const TV scale = TV(h->prm.beta_restrict / h->prm.alpha);
        with_coefs(m, [&](auto C) {
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
            const LevelArgs A = h->t->largs(m);
            launch(&h->probe, OCG_PROBE_RESTRICT, m, A.ncell, st, [&] {
                k_restrict<TV, TC, TW><<<nblk(A.ncell), BLK, 0, st>>>(A, h->t->tables(), C, U, B, scale);
            });
        });
        ck_launch("restrict");
    }
    void prolong(int m) {
        with_coefs(m, [&](auto C) {
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            const LevelArgs A = h->t->largs(m);
            launch(&h->probe, OCG_PROBE_PROLONG, m, A.ncell, st, [&] {
                k_prolong<TV, TC><<<nblk(A.ncell), BLK, 0, st>>>(A, h->t->tables(), C.d, U);
            });
        });
        ck_launch("prolong");
    }
    void coarsest(int m, bool fas) {
        with_coefs(m, [&](auto C) {
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
            const LevelArgs A = h->t->largs(m);
            int nt = (int)std::min<int64_t>(1024, (A.ncell + 31) / 32 * 32);
            launch(&h->probe, -1, m, A.ncell, st, [&] {
                k_coarsest<TV, TC, TW><<<1, nt, 0, st>>>(A, h->t->tables(), C, U, B, h->prm.nu_coarsest, fas ? 1 : 0);
            });
        });
        ck_launch("coarsest");
    }
    // Alg. 4 at level m; `fas` marks the first visit after a restriction from m+1
    void cycle(int m, bool fas) {
        if (m == H().mc) {
            coarsest(m, fas);
            return;
        }
        if (fas) fixb(m);
        for (int it = 0; it < h->prm.nu_pre; ++it) { sweep(m, 0); sweep(m, 1); }
        restrict_(m);
        for (int k = 0; k < h->prm.mu; ++k) cycle(m - 1, k == 0);
        prolong(m);
        for (int it = 0; it < h->prm.nu_post; ++it) { sweep(m, 1); sweep(m, 0); }
    }
    void run() { cycle(H().D, false); }
};

// ------------------------------------------------------------------ composite operator
// Y = A P on the tree cells (P's inner entries are overwritten with child averages);
// block partials of (p, Ap) go to part (if non-null); returns the number of partials.
template <class TO, class TC, class TW>
int64_t apply_outer(const ocg_octree* t, Coefs<TC, TW> C, TO* P, TO* Y, double* part, cudaStream_t st,
                    Probe* pr = nullptr) {
    const HostTree& H = t->H;
    for (int m = H.D; m >= 1; --m) {
        const LevelArgs A = t->largs(m);
        launch(pr, -1, m, A.ncell, st, [&] { k_avg<TO, TC><<<nblk(A.ncell), BLK, 0, st>>>(A, t->tables(), C.d, P); });
    }
    ck_launch("avg");
    int64_t nb = 0;
    for (int m = 0; m <= H.D; ++m) {
        const LevelArgs A = t->largs(m);
        launch(pr, OCG_PROBE_APPLY, m, A.ncell, st, [&] {
            k_apply<TO, TC, TW><<<nblk(A.ncell), BLK, 0, st>>>(A, t->tables(), C, P, Y, part ? part + nb : nullptr);
        });
        nb += nblk(A.ncell);
    }
    ck_launch("apply");
    return nb;
}

void finalize(ocg_hier* h, int64_t nb, int op, cudaStream_t st) {
    k_finalize<<<1, 256, 0, st>>>(h->part, nb, op, h->S, (double)h->t->H.nleaf);
    ++g_launches;
    ck_launch("finalize");
}

void ensure_work(ocg_hier* h) {
    const HostTree& H = h->t->H;
    if (!h->S) {
        h->S = dalloc<double>(S_COUNT);
        ck(cudaMallocHost((void**)&h->hS, S_COUNT * sizeof(double)), "cudaMallocHost");
    }
    int64_t need = 2 * (nblk(H.ntree) + (int64_t)(H.D + 1) + 8);
    if (h->npart < need) {
        dfree(h->part);
        h->part = nullptr;
        h->part = dalloc<double>(need);
        h->npart = need;
    }
}

void fetch_S(ocg_hier* h, cudaStream_t st) {
    ck(cudaMemcpyAsync(h->hS, h->S, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st), "copy scalars");
    ck(cudaStreamSynchronize(st), "stream sync");
}

// Alg. 1 with x0 = 0, preconditioned by one mu-cycle; TO = Krylov vector type, TV =
// cycle type, outer operator on coefficients of type TC.
template <class TO, class TV, class TC, class TW>
int pcg_run(ocg_hier* h, Coefs<TC, TW> Co, const double* b_user, double* x_user, const ocg_solve_params* sp,
            ocg_solve_stats* stats, cudaStream_t st) {
    const ocg_octree* t = h->t;
    const HostTree& H = t->H;
    const int64_t n = H.ntree;
    ensure_work(h);
    TO* x = (TO*)h->vec_of(0, n * sizeof(TO));
    TO* r = (TO*)h->vec_of(1, n * sizeof(TO));
    TO* p = (TO*)h->vec_of(2, n * sizeof(TO));
    TO* Ap = (TO*)h->vec_of(3, n * sizeof(TO));
    TV* U = (TV*)h->vec_of(4, H.ncell * sizeof(TV));
    TV* B = (TV*)h->vec_of(5, H.ncell * sizeof(TV));
    const bool ns = sp->nullspace < 0 ? h->ns_auto : sp->nullspace != 0;
    ck(cudaMemsetAsync(x, 0, n * sizeof(TO), st), "memset");
    ck(cudaMemsetAsync(r, 0, n * sizeof(TO), st), "memset");
    ck(cudaMemsetAsync(p, 0, n * sizeof(TO), st), "memset");
    ck(cudaMemsetAsync(B, 0, H.ncell * sizeof(TV), st), "memset");
    ck(cudaMemsetAsync(h->S, 0, S_COUNT * sizeof(double), st), "memset");
    const double nsv = ns ? 1.0 : 0.0;
    ck(cudaMemcpyAsync(h->S + S_NS, &nsv, sizeof(double), cudaMemcpyHostToDevice, st), "copy");
    ++g_launches;
    k_scatter<double, TO><<<nblk(H.nleaf), BLK, 0, st>>>(b_user, r, t->leaf_cell, H.nleaf);
    ck_launch("scatter");
    const unsigned gb = nblk(n);
    ++g_launches;
    k_dot<TO, TO><<<gb, BLK, 0, st>>>(r, r, n, h->part);
    finalize(h, gb, OP_BB, st);
    TV* bcast = (TV*)B;
    ++g_launches;
    k_project<TO, TV><<<gb, BLK, 0, st>>>(r, t->flags, h->S, bcast, n);
    ck_launch("project");
    fetch_S(h, st);
    const double bb = h->hS[S_BB];
    std::memset(stats, 0, sizeof(*stats));
    stats->hist[0] = 1.0;
    if (!(bb > 0.0)) {
        ck(cudaMemsetAsync(x_user, 0, H.nleaf * sizeof(double), st), "memset");
        stats->converged = 1;
        ck(cudaStreamSynchronize(st), "sync");
        return OCG_OK;
    }
    Cycle<TV> cyc{h, U, B, st};
    ck(cudaMemsetAsync(U, 0, H.ncell * sizeof(TV), st), "memset");
    cyc.run();
    ++g_launches;
    k_dot<TO, TV><<<gb, BLK, 0, st>>>(r, U, n, h->part);
    finalize(h, gb, OP_RZ0, st);
    ++g_launches;
    k_pupdate<TO, TV><<<gb, BLK, 0, st>>>(p, U, h->S, n, 1);
    ck_launch("pupdate");
    int k = 0;
    double rel = 1.0;
    int status = OCG_ENOTCONV;
    while (k < sp->max_iter) {
        const int64_t nb = apply_outer<TO, TC, TW>(t, Co, p, Ap, h->part, st, &h->probe);
        finalize(h, nb, OP_ALPHA, st);
        ++g_launches;
        k_update<TO, TV><<<gb, BLK, 0, st>>>(x, r, p, Ap, h->S, ns ? nullptr : B, n, h->part);
        ck_launch("update");
        finalize(h, gb, OP_RR, st);
        if (ns) {
            ++g_launches;
            k_project<TO, TV><<<gb, BLK, 0, st>>>(r, t->flags, h->S, B, n);
            ck_launch("project");
        }
        fetch_S(h, st);
        ++k;
        const double rr = h->hS[S_RR];
        rel = std::sqrt(std::max(rr, 0.0) / bb);
        if (k < OCG_HIST) stats->hist[k] = rel;
        if (!std::isfinite(rel)) { status = OCG_ENAN; break; }
        if (rel <= sp->tol) { status = OCG_OK; break; }
        ck(cudaMemsetAsync(U, 0, H.ncell * sizeof(TV), st), "memset");
        cyc.run();
        ++g_launches;
        k_dot<TO, TV><<<gb, BLK, 0, st>>>(r, U, n, h->part);
        finalize(h, gb, OP_BETA, st);
        ++g_launches;
        k_pupdate<TO, TV><<<gb, BLK, 0, st>>>(p, U, h->S, n, 0);
        ck_launch("pupdate");
    }
    ++g_launches;
    k_gather<TO, double><<<nblk(H.nleaf), BLK, 0, st>>>(x, x_user, t->leaf_cell, H.nleaf);
    ck_launch("gather");
    // true residual ||b - A x|| in FP64 (null-space shifted like the recursive one)
    double* xt = (double*)h->vec_of(6, n * sizeof(double));
    double* yt = (double*)h->vec_of(7, n * sizeof(double));
    ck(cudaMemsetAsync(xt, 0, n * sizeof(double), st), "memset");
    ck(cudaMemsetAsync(yt, 0, n * sizeof(double), st), "memset");
    ++g_launches;
    k_scatter<double, double><<<nblk(H.nleaf), BLK, 0, st>>>(x_user, xt, t->leaf_cell, H.nleaf);
    apply_outer<double, TC, TW>(t, Co, xt, yt, nullptr, st);
    ck(cudaMemsetAsync(xt, 0, n * sizeof(double), st), "memset");
    ++g_launches;
    k_scatter<double, double><<<nblk(H.nleaf), BLK, 0, st>>>(b_user, xt, t->leaf_cell, H.nleaf);
    ++g_launches;
    k_resid<double><<<gb, BLK, 0, st>>>(xt, yt, t->flags, n, h->part);
    finalize(h, gb, OP_RR, st);
    fetch_S(h, st);
    stats->iterations = k;
    stats->rel_res = rel;
    stats->converged = status == OCG_OK;
    stats->true_rel_res = std::sqrt(std::max(h->hS[S_RR], 0.0) / bb);
    if (status == OCG_ENOTCONV) g_err = "PCG reached max_iter before the tolerance";
    if (status == OCG_ENAN) g_err = "non-finite residual norm";
    return status;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* ocg_last_error(void) { return g_err.c_str(); }

int ocg_octree_build(const ocg_octree_desc* desc, ocg_octree** out) {
    return guard([&] {
        if (!desc || !out) throw Status(OCG_EINVAL, "null argument");
        *out = nullptr;
        std::unique_ptr<ocg_octree> t(new ocg_octree());
        try {
            build_host_tree(*desc, t->H);
        } catch (const std::runtime_error& e) {
            throw Status(OCG_EINVAL, e.what());
        }
        *out = t.release();
    });
}

void ocg_octree_destroy(ocg_octree* t) { delete t; }

int ocg_octree_counts(const ocg_octree* t, int64_t c[8]) {
    return guard([&] {
        if (!t || !c) throw Status(OCG_EINVAL, "null argument");
        const HostTree& H = t->H;
        c[0] = H.nleaf; c[1] = H.nface; c[2] = H.D; c[3] = H.mc;
        c[4] = H.ncell; c[5] = H.nt; c[6] = H.ntree; c[7] = H.noct;
    });
}

int ocg_octree_export_leaves(const ocg_octree* t, int32_t* depth, int32_t* i, int32_t* j, int32_t* k) {
    return guard([&] {
        if (!t) throw Status(OCG_EINVAL, "null octree");
        const HostTree& H = t->H;
        const size_t n = H.nleaf * sizeof(int32_t);
        if (depth) std::memcpy(depth, H.leaf_depth.data(), n);
        if (i) std::memcpy(i, H.leaf_i.data(), n);
        if (j) std::memcpy(j, H.leaf_j.data(), n);
        if (k) std::memcpy(k, H.leaf_k.data(), n);
    });
}

int ocg_octree_export_neighbours(const ocg_octree* t, int8_t* kind, int64_t* rank) {
    return guard([&] {
        if (!t) throw Status(OCG_EINVAL, "null octree");
        const HostTree& H = t->H;
        if (kind) std::memcpy(kind, H.nb_kind.data(), H.nb_kind.size());
        if (rank) std::memcpy(rank, H.nb_rank.data(), H.nb_rank.size() * sizeof(int64_t));
    });
}

int ocg_octree_export_faces(const ocg_octree* t, int32_t* axis, int32_t* depth, int32_t* i, int32_t* j,
                            int32_t* k, int64_t* minus, int64_t* plus) {
    return guard([&] {
        if (!t) throw Status(OCG_EINVAL, "null octree");
        const HostTree& H = t->H;
        const size_t n4 = H.nface * sizeof(int32_t), n8 = H.nface * sizeof(int64_t);
        if (axis) std::memcpy(axis, H.f_axis.data(), n4);
        if (depth) std::memcpy(depth, H.f_depth.data(), n4);
        if (i) std::memcpy(i, H.f_i.data(), n4);
        if (j) std::memcpy(j, H.f_j.data(), n4);
        if (k) std::memcpy(k, H.f_k.data(), n4);
        if (minus) std::memcpy(minus, H.f_minus.data(), n8);
        if (plus) std::memcpy(plus, H.f_plus.data(), n8);
    });
}

int ocg_octree_export_level(const ocg_octree* t, int32_t m, int64_t* n, int32_t* i, int32_t* j, int32_t* k,
                            int8_t* leaf) {
    return guard([&] {
        if (!t || !n) throw Status(OCG_EINVAL, "null argument");
        const HostTree& H = t->H;
        if (m < H.mc || m > H.D) throw Status(OCG_EINVAL, "level out of range");
        const LevelMeta& l = H.L(m);
        int64_t c = 0;
        for (int64_t g = l.off; g < l.off + l.ncell; ++g) {
            if (!(H.cell_flags[g] & 2)) continue;
            if (i) {
                int64_t a, b, d;
                H.cell_coords(m, g, a, b, d);
                i[c] = (int32_t)a; j[c] = (int32_t)b; k[c] = (int32_t)d;
                if (leaf) leaf[c] = (int8_t)(H.cell_flags[g] & 1);
            }
            ++c;
        }
        *n = c;
    });
}

int ocg_setup_hierarchy(const ocg_octree* t, const float* beta, const int32_t bc[6], const ocg_mg_params* prm,
                        void* stream, ocg_hier** out) {
    return guard([&] {
        if (!t || !beta || !bc || !prm || !out) throw Status(OCG_EINVAL, "null argument");
        *out = nullptr;
        if (prm->mu < 1 || prm->mu > 4 || prm->nu_pre < 0 || prm->nu_post < 0 || prm->nu_coarsest < 0 ||
            !(prm->alpha > 0) || !std::isfinite(prm->beta_restrict))
            throw Status(OCG_EINVAL, "invalid multigrid parameters");
        if (prm->coef_dtype != OCG_F64 && prm->coef_dtype != OCG_F32) throw Status(OCG_EINVAL, "coef_dtype");
        if (prm->bf16_coarse && prm->coef_dtype != OCG_F32) throw Status(OCG_EINVAL, "bf16_coarse needs F32");
        for (int q = 0; q < 6; ++q)
            if (bc[q] != OCG_BC_NEUMANN && bc[q] != OCG_BC_DIRICHLET) throw Status(OCG_EINVAL, "bc code");
        cudaStream_t st = (cudaStream_t)stream;
        const HostTree& H = t->H;
        t->upload();
        std::unique_ptr<ocg_hier> h(new ocg_hier());
        h->t = t;
        h->prm = *prm;
        bool ns = true;
        for (int q = 0; q < 6; ++q) {
            h->bc[q] = bc[q];
            if (bc[q] == OCG_BC_DIRICHLET) ns = false;
        }
        h->ns_auto = ns;
        for (int q = 0; q < 4; ++q) h->c64[q] = dalloc<double>(H.ncell);
        const int64_t ntw = 24 * std::max<int64_t>(H.nt, 1);
        h->tw64 = dalloc<double>(ntw);
        for (int q = 0; q < 4; ++q) ck(cudaMemsetAsync(h->c64[q], 0, H.ncell * sizeof(double), st), "memset");
        ck(cudaMemsetAsync(h->tw64, 0, ntw * sizeof(double), st), "memset");
        // c64[1..3] are contiguous views for the kernels' [3][ncell] indexing: allocate
        // one block instead
        double* cm = dalloc<double>(3 * H.ncell);
        ck(cudaMemsetAsync(cm, 0, 3 * H.ncell * sizeof(double), st), "memset");
        std::vector<double> hd(H.D + 1);
        for (int d = 0; d <= H.D; ++d) hd[d] = 1.0 / (double)((int64_t)H.n0 << d);
        double* dh = dupload(hd);
        int* derr = dalloc<int>(1);
        ck(cudaMemsetAsync(derr, 0, sizeof(int), st), "memset");
        k_face_scatter<<<nblk(H.nface), BLK, 0, st>>>(beta, t->fslot, t->fkind, t->fdepth, dh, H.nface, cm,
                                                     h->tw64, derr);
        ck_launch("face scatter");
        LevelTab LT{};
        LT.mc = H.mc;
        for (int m = H.mc; m <= H.D; ++m) {
            LT.off[m - H.mc] = H.L(m).off;
            LT.h[m - H.mc] = H.L(m).h;
        }
        k_leaf_gather<<<nblk(H.nleaf), BLK, 0, st>>>(t->leaf_cell, t->level, t->tables(), LT,
                                                    make_int4(bc[0], bc[1], bc[2], bc[3]), make_int2(bc[4], bc[5]),
                                                    H.nleaf, H.ncell, h->c64[0], cm, h->tw64);
        ck_launch("leaf gather");
        for (int m = H.D; m > H.mc; --m) {
            const LevelArgs A = t->largs(m);
            k_coarsen<<<nblk(A.ncell / 8), BLK, 0, st>>>(A, t->tables(), prm->alpha, h->c64[0], cm, H.ncell);
            ck_launch("coarsen");
        }
        for (int q = 0; q < 3; ++q)
            ck(cudaMemcpyAsync(h->c64[q + 1], cm + q * H.ncell, H.ncell * sizeof(double), cudaMemcpyDeviceToDevice, st),
               "copy");
        int herr = 0;
        ck(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
        ck(cudaStreamSynchronize(st), "setup sync");
        dfree(cm); dfree(dh); dfree(derr);
        if (herr) throw Status(OCG_EINVAL, "face beta must be finite and >= 0");
        if (prm->coef_dtype == OCG_F32) {
            for (int q = 0; q < 4; ++q) {
                h->c32[q] = dalloc<float>(H.ncell);
                k_convert<float><<<nblk(H.ncell), BLK, 0, st>>>(h->c64[q], h->c32[q], H.ncell);
                if (prm->bf16_coarse) {
                    h->c16[q] = dalloc<__nv_bfloat16>(H.ncell);
                    k_convert<__nv_bfloat16><<<nblk(H.ncell), BLK, 0, st>>>(h->c64[q], h->c16[q], H.ncell);
                }
            }
            h->tw32 = dalloc<float>(ntw);
            k_convert<float><<<nblk(ntw), BLK, 0, st>>>(h->tw64, h->tw32, ntw);
            ck_launch("convert");
            ck(cudaStreamSynchronize(st), "setup sync");
            for (int q = 0; q < 4; ++q) { dfree(h->c64[q]); h->c64[q] = nullptr; }
            dfree(h->tw64);
            h->tw64 = nullptr;
        }
        *out = h.release();
    });
}

void ocg_hier_destroy(ocg_hier* h) { delete h; }

int ocg_hier_export_coefs(const ocg_hier* h, int32_t m, double* c, double* cx, double* cy, double* cz) {
    return guard([&] {
        if (!h) throw Status(OCG_EINVAL, "null hierarchy");
        const HostTree& H = h->t->H;
        if (m < H.mc || m > H.D) throw Status(OCG_EINVAL, "level out of range");
        const LevelMeta& l = H.L(m);
        double* outs[4] = {c, cx, cy, cz};
        std::vector<double> buf(l.ncell);
        std::vector<float> bf(l.ncell);
        for (int q = 0; q < 4; ++q) {
            if (!outs[q]) continue;
            if (h->c64[q]) {
                ck(cudaMemcpy(buf.data(), h->c64[q] + l.off, l.ncell * sizeof(double), cudaMemcpyDeviceToHost), "copy");
            } else {
                ck(cudaMemcpy(bf.data(), h->c32[q] + l.off, l.ncell * sizeof(float), cudaMemcpyDeviceToHost), "copy");
                for (int64_t i = 0; i < l.ncell; ++i) buf[i] = bf[i];
            }
            int64_t n = 0;
            for (int64_t g = 0; g < l.ncell; ++g)
                if (H.cell_flags[l.off + g] & 2) outs[q][n++] = buf[g];
        }
    });
}

int ocg_apply_A(ocg_hier* h, int32_t dtype, const void* x, void* y, int32_t transpose, void* stream) {
    return guard([&] {
        if (!h || !x || !y) throw Status(OCG_EINVAL, "null argument");
        if (transpose) throw Status(OCG_EINVAL, "transpose is not available in this version");
        cudaStream_t st = (cudaStream_t)stream;
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        auto run = [&](auto* tag, auto C) {
            using TO = std::remove_pointer_t<decltype(tag)>;
            using CC = decltype(C);
            using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::d)>>;
            using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
            TO* P = (TO*)h->vec_of(6, H.ntree * sizeof(TO));
            TO* Y = (TO*)h->vec_of(7, H.ntree * sizeof(TO));
            ck(cudaMemsetAsync(P, 0, H.ntree * sizeof(TO), st), "memset");
            k_scatter<TO, TO><<<nblk(H.nleaf), BLK, 0, st>>>((const TO*)x, P, t->leaf_cell, H.nleaf);
            apply_outer<TO, TC, TW>(t, C, P, Y, nullptr, st);
            k_gather<TO, TO><<<nblk(H.nleaf), BLK, 0, st>>>(Y, (TO*)y, t->leaf_cell, H.nleaf);
            ck_launch("apply_A");
        };
        if (dtype == OCG_F64) {
            if (h->c64[0]) run((double*)nullptr, h->C64());
            else run((double*)nullptr, h->C32());
        } else if (dtype == OCG_F32) {
            if (h->c64[0]) run((float*)nullptr, h->C64());
            else run((float*)nullptr, h->C32());
        } else {
            throw Status(OCG_EINVAL, "dtype");
        }
    });
}

int ocg_vcycle(ocg_hier* h, int32_t dtype, const void* r, void* z, void* stream) {
    return guard([&] {
        if (!h || !r || !z) throw Status(OCG_EINVAL, "null argument");
        cudaStream_t st = (cudaStream_t)stream;
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        auto run = [&](auto* tag) {
            using TV = std::remove_pointer_t<decltype(tag)>;
            TV* U = (TV*)h->vec_of(4, H.ncell * sizeof(TV));
            TV* B = (TV*)h->vec_of(5, H.ncell * sizeof(TV));
            ck(cudaMemsetAsync(U, 0, H.ncell * sizeof(TV), st), "memset");
            ck(cudaMemsetAsync(B, 0, H.ncell * sizeof(TV), st), "memset");
            k_scatter<TV, TV><<<nblk(H.nleaf), BLK, 0, st>>>((const TV*)r, B, t->leaf_cell, H.nleaf);
            Cycle<TV> cyc{h, U, B, st};
            cyc.run();
            k_gather<TV, TV><<<nblk(H.nleaf), BLK, 0, st>>>(U, (TV*)z, t->leaf_cell, H.nleaf);
            ck_launch("vcycle");
        };
        if (dtype == OCG_F64) {
            if (!h->c64[0]) throw Status(OCG_EINVAL, "F64 cycle needs coef_dtype F64");
            run((double*)nullptr);
        } else if (dtype == OCG_F32) {
            if (!h->c32[0]) throw Status(OCG_EINVAL, "F32 cycle needs coef_dtype F32");
            run((float*)nullptr);
        } else {
            throw Status(OCG_EINVAL, "dtype");
        }
    });
}

int ocg_pcg_solve(ocg_hier* h, const double* b, double* x, const ocg_solve_params* sp, ocg_solve_stats* stats,
                  void* stream) {
    int status = OCG_OK;
    int g = guard([&] {
        if (!h || !b || !x || !sp || !stats) throw Status(OCG_EINVAL, "null argument");
        if (!(sp->tol > 0) || sp->max_iter < 0) throw Status(OCG_EINVAL, "tol / max_iter");
        cudaStream_t st = (cudaStream_t)stream;
        switch (sp->precision) {
            case OCG_PREC_FP64:
                if (!h->c64[0]) throw Status(OCG_EINVAL, "FP64 solve needs coef_dtype F64");
                status = pcg_run<double, double>(h, h->C64(), b, x, sp, stats, st);
                break;
            case OCG_PREC_FP32:
                if (!h->c32[0]) throw Status(OCG_EINVAL, "FP32 solve needs coef_dtype F32");
                status = pcg_run<float, float>(h, h->C32(), b, x, sp, stats, st);
                break;
            case OCG_PREC_MIXED:
                if (!h->c32[0]) throw Status(OCG_EINVAL, "mixed solve needs coef_dtype F32");
                status = pcg_run<double, float>(h, h->C32(), b, x, sp, stats, st);
                break;
            default:
                throw Status(OCG_EINVAL, "precision");
        }
    });
    return g != OCG_OK ? g : status;
}

}  // extern "C"

extern "C" {

int ocg_probe_set(ocg_hier* h, int32_t kind, int32_t level) {
    return guard([&] {
        if (!h) throw Status(OCG_EINVAL, "null hierarchy");
        if (kind < OCG_PROBE_OFF || kind > OCG_PROBE_APPLY) throw Status(OCG_EINVAL, "probe kind");
        h->probe.kind = kind;
        h->probe.level = level;
        h->probe.used = 0;
    });
}

int ocg_probe_read(ocg_hier* h, void* stream, int64_t* launches, double* total_ms, int64_t* cells) {
    return guard([&] {
        if (!h || !launches || !total_ms || !cells) throw Status(OCG_EINVAL, "null argument");
        ck(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
        double tot = 0.0;
        for (int64_t q = 0; q + 1 < h->probe.used; q += 2) {
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, h->probe.ev[q], h->probe.ev[q + 1]), "cudaEventElapsedTime");
            tot += ms;
        }
        *launches = h->probe.used / 2;
        *total_ms = tot;
        *cells = h->probe.cells;
        h->probe.used = 0;
    });
}

int ocg_launch_count(int64_t* n) {
    return guard([&] {
        if (!n) throw Status(OCG_EINVAL, "null argument");
        *n = g_launches.load();
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Operator apply without allocation: the two internal-layout work vectors (the input
// scattered to cell order, and the output in cell order) live in this fixed array.
namespace {
static __device__ __align__(256) float g_noalloc_scratch[2 * (int64_t)OCG_NOALLOC_MAX_CELLS];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[256] = {};   // device address of g_noalloc_scratch per device ordinal

float* noalloc_scratch() {
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 256) throw Status(OCG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        ck(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = (float*)p;
    }
    return g_noalloc_ptr[dev];
}
}  // namespace

extern "C" int ocg_apply_A_f32_noalloc(ocg_hier* h, const float* x, float* y, void* stream) {
    return guard([&] {
        if (!h || !x || !y) throw Status(OCG_EINVAL, "null argument");
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        if (!t->on_device) throw Status(OCG_ESTATE, "octree tables are not on the device");
        if (H.ntree > (int64_t)OCG_NOALLOC_MAX_CELLS)
            throw Status(OCG_EINVAL, "tree has " + std::to_string(H.ntree) + " cells; the allocation-free apply "
                                     "accepts at most " + std::to_string((int64_t)OCG_NOALLOC_MAX_CELLS));
        cudaStream_t st = (cudaStream_t)stream;
        float* base = noalloc_scratch();
        float* P = base;
        float* Y = base + OCG_NOALLOC_MAX_CELLS;
        // cells that are not leaves are overwritten by child averages before use; clear
        // anyway so no value of an earlier call can leak into this one
        ck(cudaMemsetAsync(P, 0, H.ntree * sizeof(float), st), "memset");
        k_scatter<float, float><<<nblk(H.nleaf), BLK, 0, st>>>(x, P, t->leaf_cell, H.nleaf);
        ck_launch("scatter");
        if (h->c64[0]) apply_outer<float, double, double>(t, h->C64(), P, Y, nullptr, st);
        else apply_outer<float, float, float>(t, h->C32(), P, Y, nullptr, st);
        k_gather<float, float><<<nblk(H.nleaf), BLK, 0, st>>>(Y, y, t->leaf_cell, H.nleaf);
        ck_launch("gather");
        g_launches += 2;
    });
}
