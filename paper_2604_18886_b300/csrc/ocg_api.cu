// libocg: C ABI, hierarchy set-up, the mu-cycle driver and the PCG loop.
// Every arithmetic step of the solve runs in the kernels of kernels.cuh; this file only
// allocates device memory, uploads the octree tables and sequences launches.  The PCG
// loop is captured once per (hierarchy, precision, null-space mode) into a CUDA graph
// whose iterations run under a conditional WHILE node: the convergence test of Alg. 1
// is evaluated by the reduction kernel that forms ||r||, so a solve needs no host round
// trip per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ocg.h"
#include "batch.cuh"
#include "kernels.cuh"
#include "octet.cuh"
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
        cudaGetLastError();   // clear a non-sticky error so later launch checks do not see it
        if (e == cudaErrorMemoryAllocation) throw Status(OCG_ENOMEM, std::string(what) + ": out of device memory");
        throw Status(OCG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void ck_launch(const char* what) { ck(cudaGetLastError(), what); }

// Device allocations go through cudaMalloc or the caller's hooks (ocg_set_allocator); a
// block is freed by the allocator that made it, whatever is set at that time.
struct AllocHooks {
    ocg_alloc_fn alloc = nullptr;
    ocg_free_fn free = nullptr;
    void* ctx = nullptr;
};
std::mutex g_alloc_mu;
AllocHooks g_hooks;
std::unordered_map<void*, AllocHooks> g_hooked;   // blocks made through the hooks

template <class T>
T* dalloc(int64_t n) {
    void* p = nullptr;
    if (n <= 0) n = 1;
    const size_t bytes = (size_t)n * sizeof(T);
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_hooks.alloc) {
        p = g_hooks.alloc(bytes, g_hooks.ctx);
        if (!p) throw Status(OCG_ENOMEM, "allocator hook returned NULL");
        if (reinterpret_cast<uintptr_t>(p) % 256) {
            g_hooks.free(p, g_hooks.ctx);
            throw Status(OCG_EINVAL, "allocator hook returned memory not aligned to 256 bytes");
        }
        g_hooked[p] = g_hooks;
        return (T*)p;
    }
    ck(cudaMalloc(&p, bytes), "cudaMalloc");
    return (T*)p;
}

template <class T, class A>
T* dupload(const std::vector<T, A>& v) {
    T* p = dalloc<T>((int64_t)v.size());
    if (!v.empty()) ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
    return p;
}

void dfree(void* p) {
    if (!p) return;
    AllocHooks hk;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_hooked.find(p);
        if (it == g_hooked.end()) {
            cudaFree(p);
            return;
        }
        hk = it->second;
        g_hooked.erase(it);
    }
    hk.free(p, hk.ctx);
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

// Kernel launch with the programmatic-serialization attribute (see pdl_enter); OCG_PDL=0
// in the environment launches without it.
inline bool pdl_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("OCG_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    if (e != cudaSuccess) throw Status(OCG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
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
        record(ev[used], st);
    }
    void end(cudaStream_t st) {
        record(ev[used + 1], st);
        used += 2;
    }
    // under stream capture a plain record only joins streams; an external record becomes
    // an event-record node that timestamps like a stream record
    static void record(cudaEvent_t e, cudaStream_t st) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        ck(cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
        if (cs == cudaStreamCaptureStatusActive)
            ck(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
        else
            ck(cudaEventRecord(e, st), "cudaEventRecord");
    }
};

// Launch context: stream, probe (eager launches only; null while capturing) and a
// counter of the kernels issued through it.
struct Ctx {
    cudaStream_t st;
    Probe* probe;
    int64_t count;
};

template <class F>
void launch(Ctx& c, int kind, int m, int64_t cells, F&& f) {
    const bool p = c.probe && c.probe->on(kind, m);
    if (p) {
        c.probe->cells = cells;
        c.probe->begin(c.st);
    }
    f();
    ++c.count;
    if (p) c.probe->end(c.st);
}

}  // namespace

struct ocg_octree {
    HostTree H;
    // device copies of the tables, uploaded by the first hierarchy set-up
    mutable bool on_device = false;
    mutable int device = -1;   // CUDA device ordinal that holds the tables once uploaded
    mutable int32_t *nbr = nullptr, *oct_parent = nullptr, *child_oct = nullptr, *trec = nullptr,
                    *leaf_cell = nullptr;
    mutable uint8_t* flags = nullptr;
    mutable int8_t* level = nullptr;
    mutable int64_t* fslot = nullptr;
    mutable uint8_t* fkind = nullptr;
    mutable int8_t* fdepth = nullptr;

    void upload() const {
        int dev = 0;
        ck(cudaGetDevice(&dev), "cudaGetDevice");
        if (on_device) {
            if (dev != device)
                throw Status(OCG_EINVAL, "the octree's tables are on device " + std::to_string(device) +
                                         ", the current device is " + std::to_string(dev));
            return;
        }
        device = dev;
        nbr = dupload(H.nbr);
        oct_parent = dupload(H.oct_parent);
        child_oct = dupload(H.child_oct);
        trec = dupload(H.trec);
        leaf_cell = dupload(H.leaf_cell);
        flags = dupload(H.cell_flags);
        level = dupload(H.cell_level);
        fslot = dupload(H.f_slot);
        fkind = dupload(H.f_kind);
        fdepth = dupload(H.f_depth);
        on_device = true;
    }
    Tables tables() const { return Tables{nbr, oct_parent, child_oct, trec, (int)H.noct, (int)H.nt}; }
    LevelArgs largs(int m) const { return LevelArgs{(int)H.L(m).off, (int)H.L(m).ncell, H.L(m).ni}; }

    // adjoint tables (topology only), built on first use
    mutable std::mutex adj_mu;
    mutable bool adj_ready = false;
    mutable int n_tcoarse = 0, n_tdesc = 0;
    mutable int32_t *t_oct = nullptr, *tcoarse = nullptr, *tdesc = nullptr, *fminus = nullptr, *fplus = nullptr;
    mutable std::vector<int> tc_lo, tc_hi;   // per tree level m: the range of tcoarse in level m
    void upload_adjoint() const {
        std::lock_guard<std::mutex> lk(adj_mu);
        if (adj_ready) return;
        AdjointTopology at;
        build_adjoint_topology(H, at);
        n_tcoarse = (int)at.tcoarse.size();
        n_tdesc = (int)at.tdesc.size();
        tc_lo.assign(H.D + 1, 0);
        tc_hi.assign(H.D + 1, 0);
        for (int m = 0; m <= H.D; ++m) {
            const int64_t a = H.L(m).off, b = a + H.L(m).ncell;
            tc_lo[m] = (int)(std::lower_bound(at.tcoarse.begin(), at.tcoarse.end(), a) - at.tcoarse.begin());
            tc_hi[m] = (int)(std::lower_bound(at.tcoarse.begin(), at.tcoarse.end(), b) - at.tcoarse.begin());
        }
        t_oct = dupload(H.t_oct);
        tcoarse = dupload(at.tcoarse);
        tdesc = dupload(at.tdesc);
        fminus = dupload(H.f_minus);
        fplus = dupload(H.f_plus);
        adj_ready = true;
    }
    ~ocg_octree() {
        dfree(nbr); dfree(oct_parent); dfree(child_oct); dfree(trec); dfree(leaf_cell);
        dfree(flags); dfree(level); dfree(fslot); dfree(fkind); dfree(fdepth);
        dfree(t_oct); dfree(tcoarse); dfree(tdesc); dfree(fminus); dfree(fplus);
    }
};

constexpr int TAIL_NONE = 1 << 20;   // larger than any level index

struct GraphSolve {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t outer_kernels = 0;   // kernels outside the WHILE body
    int64_t body_kernels = 0;    // kernels per WHILE iteration
};

struct ocg_hier {
    const ocg_octree* t = nullptr;
    int device = -1;   // CUDA device ordinal current at set-up; every later call must run there
    ocg_mg_params prm{};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    bool ns_auto = false;
    double* c64[4] = {nullptr, nullptr, nullptr, nullptr};
    double* tw64 = nullptr;
    double* tseed = nullptr;   // adjoint: per tree cell, the a_P weight sums of the T faces
    float* c32[4] = {nullptr, nullptr, nullptr, nullptr};
    float* tw32 = nullptr;
    __nv_bfloat16* c16[4] = {nullptr, nullptr, nullptr, nullptr};   // [0] unused: see d16
    float* d16 = nullptr;         // conservative FP32 diagonal of the BF16 set
    float* rem32 = nullptr;       // FP32 sets: diagonal remainder of the tree cells (k_remainder)
    // work space, allocated once at set-up at the widest type so a captured graph keeps
    // valid pointers: x, r, p, Ap, bt (b in cell order), xt, yt over the tree cells;
    // U, B over all cells
    double *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *bt = nullptr, *xt = nullptr, *yt = nullptr;
    double *U = nullptr, *B = nullptr;
    double* S = nullptr;       // device scalars
    double* hS = nullptr;      // pinned host mirror
    double* part = nullptr;    // block partials
    unsigned* cnt = nullptr;   // reduction arrival counter
    Probe probe;
    int red_blocks = 296;         // grid of the grid-stride reductions (2 per SM)
    int sweep_form[MAXLEV * 2];   // per level (index m - mc): OCG_SWEEP_OCTET / _CELL / _QUAD
    double tune_us[MAXLEV * 2][4];
    // coarse tail: uniform levels run in one shared-memory CTA, per cycle value type
    int tail_top[2] = {TAIL_NONE, TAIL_NONE};   // [float, double]
    size_t tail_smem[2] = {0, 0};
    TailArgs tail_args[2];
    int* tail_sched = nullptr;    // device copies of the tail pass schedules (float, double)
    int* tail_sched2 = nullptr;
    cudaStream_t cap = nullptr;   // private stream for graph capture
    GraphSolve graphs[3][3][2][2];   // [A by PCG, A^T by PCG, A^T by BiCGStab][precision][null space][warm]
    float* beta = nullptr;        // copy of the face fractions (transposed operator)
    // BiCGStab vectors over the tree cells (adjoint solves), allocated on first use
    double *rhat = nullptr, *s = nullptr, *tv = nullptr, *ph = nullptr, *sh = nullptr;
    // transposed cycle scratch over all cells, allocated on first use
    double *Xc = nullptr, *UST = nullptr;
    double* Tacc = nullptr;   // [6][nt]: per T record and face, the coarser leaf's share (zero between uses)

    Coefs<double, double> C64() const { return {c64[0], c64[1], c64[2], c64[3], tw64}; }
    Coefs<float, float> C32() const { return {c32[0], c32[1], c32[2], c32[3], tw32}; }
    Coefs<__nv_bfloat16, float> C16() const { return {d16, c16[1], c16[2], c16[3], tw32}; }

    ~ocg_hier() {
        for (auto& tr : graphs)
            for (auto& row : tr)
                for (auto& pair : row)
                    for (auto& gs : pair) {
                        if (gs.exec) cudaGraphExecDestroy(gs.exec);
                        if (gs.graph) cudaGraphDestroy(gs.graph);
                    }
        for (double* v : {rhat, s, tv, ph, sh, Xc, UST, Tacc}) dfree(v);
        dfree(beta);
        dfree(tseed);
        if (cap) cudaStreamDestroy(cap);
        for (int i = 0; i < 4; ++i) { dfree(c64[i]); dfree(c32[i]); dfree(c16[i]); }
        dfree(d16);
        dfree(rem32);
        dfree(tw64); dfree(tw32); dfree(S); dfree(part); dfree(cnt); dfree(tail_sched); dfree(tail_sched2);
        if (hS) cudaFreeHost(hS);
        for (double* v : {x, r, p, Ap, bt, xt, yt, U, B}) dfree(v);
    }
};

namespace {

// Recursions into level m per visit of level m + 1: mu, or 1 when mu_min_cells is set and
// level m has fewer real cells (padding excluded).
int mu_at(const ocg_hier* h, int m) {
    const HostTree& H = h->t->H;
    if (h->prm.mu <= 1 || h->prm.mu_min_cells <= 0) return h->prm.mu;
    const LevelMeta& L = H.L(m);
    const int64_t cells = m >= 0 ? L.ncell : (int64_t)L.N * L.N * L.N;
    return cells >= h->prm.mu_min_cells ? h->prm.mu : 1;
}

// The tail is the longest run of the coarsest levels m < 0, up to level max_top, whose
// shared-memory image (u, b and four coefficients per cell) fits in 200 KB.
void choose_tail(ocg_hier* h, int which, size_t vbytes, int max_top = -1) {
    const HostTree& H = h->t->H;
    int top = TAIL_NONE;
    int64_t cells = 0;
    for (int m = H.mc; m < 0 && m <= max_top; ++m) {
        const int64_t c = cells + H.L(m).ncell;
        if ((size_t)c * 6 * vbytes > 200 * 1024 || m - H.mc + 1 > MAXLEV) break;
        cells = c;
        top = m;
    }
    h->tail_top[which] = top;
    if (top == TAIL_NONE) return;
    TailArgs& A = h->tail_args[which];
    std::memset(&A, 0, sizeof(A));
    A.nlev = top - H.mc + 1;
    int sb = 0;
    for (int li = 0; li < A.nlev; ++li) {
        const int m = top - li;
        A.L[li].off = (int)H.L(m).off;
        A.L[li].ni = H.L(m).ni;
        A.L[li].sbase = sb;
        sb += (int)H.L(m).ncell;
    }
    A.ncell = sb;
    A.up_off = (int)H.L(top + 1).off;
    A.up_ni = H.L(top + 1).ni;
    // expand the sub-cycle (Alg. 4 over the tail levels) into a flat pass schedule
    std::vector<int> sch;
    const ocg_mg_params& P = h->prm;
    auto emit = [&](int li, int kind) { sch.push_back(8 * li + kind); };
    std::function<void(int, bool)> rec = [&](int li, bool fas) {
        if (fas) emit(li, TP_FIXB);
        if (li == A.nlev - 1) {
            const int half = P.nu_coarsest / 2;
            for (int it = 0; it < half; ++it) { emit(li, 0); emit(li, 1); }
            for (int it = half; it < P.nu_coarsest; ++it) { emit(li, 1); emit(li, 0); }
            return;
        }
        for (int it = 0; it < P.nu_pre; ++it) { emit(li, 0); emit(li, 1); }
        emit(li, TP_RESTRICT);
        const int mu = mu_at(h, top - (li + 1));
        for (int k = 0; k < mu; ++k) rec(li + 1, k == 0);
        emit(li, TP_PROLONG);
        for (int it = 0; it < P.nu_post; ++it) { emit(li, 1); emit(li, 0); }
    };
    rec(0, false);
    int* dev = dupload(sch);
    if (which == 0) {
        dfree(h->tail_sched);
        h->tail_sched = dev;
    } else {
        dfree(h->tail_sched2);
        h->tail_sched2 = dev;
    }
    A.sched = dev;
    A.nsched = (int)sch.size();
    h->tail_smem[which] = (size_t)sb * 6 * vbytes;
}

// Real (non-padding) cells of level m in the level's Morton order.
void export_faces(const HostTree& H, int64_t first, int64_t count, int32_t* axis, int32_t* depth, int32_t* i,
                  int32_t* j, int32_t* k, int64_t* minus, int64_t* plus) {
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < count; ++q) {
        const int64_t f = first + q;
        if (axis) axis[q] = H.f_axis[f];
        if (depth) depth[q] = H.f_depth[f];
        if (i || j || k) {
            int32_t a, b, c;
            face_plus_cell(H, f, a, b, c);
            if (i) i[q] = a;
            if (j) j[q] = b;
            if (k) k[q] = c;
        }
        if (minus) minus[q] = H.f_minus[f];
        if (plus) plus[q] = H.f_plus[f];
    }
}

std::vector<int64_t> level_cells_morton(const HostTree& H, int m) {
    const LevelMeta& l = H.L(m);
    std::vector<std::pair<uint64_t, int64_t>> v;
    for (int64_t g = l.off; g < l.off + l.ncell; ++g) {
        if (!(H.cell_flags[g] & 2)) continue;
        int64_t a, b, d;
        H.cell_coords(m, g, a, b, d);
        v.push_back({morton3(a, b, d), g});
    }
    std::sort(v.begin(), v.end());
    std::vector<int64_t> out(v.size());
    for (size_t q = 0; q < v.size(); ++q) out[q] = v[q].second;
    return out;
}

// ------------------------------------------------------------------ mu-cycle driver
template <class CC>
struct CoefTypes {
    using TC = std::remove_const_t<std::remove_pointer_t<decltype(CC::cx)>>;
    using TW = std::remove_const_t<std::remove_pointer_t<decltype(CC::tw)>>;
};

template <class TV>
struct Cycle {
    ocg_hier* h;
    TV* U;
    TV* B;
    Ctx& c;
    bool skip_first = false;   // the first colour-0 sweep of the finest level was fused into
                               // the Krylov update (FirstSweep), which also zeroed u

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
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, -1, m, A.ncell, [&] {
                launch_k(k_osweep<TV, TC, TW, 2>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, B, 0);
            });
        });
        ck_launch("fixb");
    }
    void sweep(int m, int colour, int prolong, int form = -2) {
        if (skip_first && m == H().D && colour == 0) {
            skip_first = false;
            return;
        }
        if (form == -2) form = h->sweep_form[m - H().mc];
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_SWEEP, m, A.ncell, [&] {
                if (form == OCG_SWEEP_CELL)
                    launch_k(k_csweep<TV, TC, TW>, nblk(A.ncell), BLK, 0, c.st, A, h->t->tables(), C, U, B, colour, prolong);
                else if (form == OCG_SWEEP_QUAD)
                    launch_k(k_qsweep<TV, TC, TW>, nblk(A.ncell / 4), BLK, 0, c.st, A, h->t->tables(), C, U, B, colour, prolong);
                else if (form == OCG_SWEEP_TILE)
                    launch_k(k_tsweep<TV, TC, TW>, nblk(A.ncell / 8, TBLK), TBLK, 0, c.st, A, h->t->tables(), C, U, B, colour,
                                                                                  prolong);
                else if (colour)
                    launch_k(k_osweep<TV, TC, TW, 1>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, B, prolong);
                else
                    launch_k(k_osweep<TV, TC, TW, 0>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, B, prolong);
            });
        });
        ck_launch("sweep");
    }
    void restrict_(int m) {
        const TV scale = TV(h->prm.beta_restrict / h->prm.alpha);
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_RESTRICT, m, A.ncell, [&] {
                launch_k(k_orestrict<TV, TC, TW>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, B, scale);
            });
        });
        ck_launch("restrict");
    }
    void prolong(int m) {
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_PROLONG, m, A.ncell, [&] {
                launch_k(k_oprolong<TV, std::remove_const_t<std::remove_pointer_t<decltype(C.d)>>>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C.d, U);
            });
        });
        ck_launch("prolong");
    }
    void coarsest(int m, bool fas, bool prolong_up) {
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            const int nt = (int)std::min<int64_t>(256, (A.ncell / 8 + 31) / 32 * 32);
            launch(c, -1, m, A.ncell, [&] {
                launch_k(k_ocoarsest<TV, TC, TW>, 1, nt, 0, c.st, A, h->t->tables(), C, U, B, h->prm.nu_coarsest,
                                                           fas ? 1 : 0, prolong_up ? 1 : 0);
            });
        });
        ck_launch("coarsest");
    }
    static constexpr int W = std::is_same<TV, double>::value ? 1 : 0;
    // The shared-memory tail; its prolongation onto the uniform level above runs as a
    // separate grid-wide launch (k_oprolong, the same arithmetic), which one CTA would take
    // several memory latencies for.
    void tail(bool fas, bool prolong_up) {
        const int m = h->tail_top[W];
        TailArgs A = h->tail_args[W];
        A.fas = fas ? 1 : 0;
        A.prolong = 0;
        const TV scale = TV(h->prm.beta_restrict / h->prm.alpha);
        const size_t sm = h->tail_smem[W];
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            ck(cudaFuncSetAttribute(k_otail<TV, TC, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
               "cudaFuncSetAttribute");
            // the widest pass is a colour sweep of the top level: 4 cells per octet
            const int noct = A.L[0].ni * A.L[0].ni * A.L[0].ni;
            const int nt = std::min(sizeof(TV) == 8 ? 256 : 1024, (4 * noct + 31) / 32 * 32);
            launch(c, OCG_PROBE_TAIL, m, A.ncell, [&] {
                launch_k(k_otail<TV, TC, TW>, 1, nt, sm, c.st, A, h->t->tables(), C, U, B, scale);
            });
        });
        ck_launch("tail");
        if (prolong_up) prolong(m + 1);
    }
    // Alg. 4 at level m.  fas: first visit after a restriction from m+1 (complete the
    // FAS right-hand side); prolong_up: the last visit, whose final operation prolongs
    // onto level m+1.
    void cycle(int m, bool fas, bool prolong_up) {
        if (m == h->tail_top[W]) { tail(fas, prolong_up); return; }
        if (m == H().mc) { coarsest(m, fas, prolong_up); return; }
        if (fas) fixb(m);
        for (int it = 0; it < h->prm.nu_pre; ++it) { sweep(m, 0, 0); sweep(m, 1, 0); }
        restrict_(m);
        const int mu = mu_at(h, m - 1);
        for (int k = 0; k < mu; ++k) cycle(m - 1, k == 0, k == mu - 1);
        const int np = h->prm.nu_post;
        for (int it = 0; it < np; ++it) {
            sweep(m, 1, 0);
            sweep(m, 0, (it == np - 1 && prolong_up) ? 1 : 0);
        }
        if (np == 0 && prolong_up) prolong(m + 1);
    }
    void run() { cycle(H().D, false, false); }
};

// The Krylov update can take over the first step of the next cycle (FirstSweep) when that
// step is a colour-0 sweep of the finest level: an FP32 cycle whose finest level is swept
// by launches (not the coarsest level, not inside the shared-memory tail), nu_pre >= 1.
inline bool first_sweep_fusable(const ocg_hier* h) {
    const HostTree& H = h->t->H;
    return h->c32[0] && h->prm.nu_pre >= 1 && H.D != H.mc && H.D != h->tail_top[0];
}

OMultiLevel tree_levels(const HostTree& H);

// ------------------------------------------------------------- transposed mu-cycle
// M^T for the adjoint system (no counterpart in the paper): the transposes of the steps of
// Cycle, in reverse order, on the adjoint state (ubar in U, bbar in B).  Input: ubar = z on
// the leaves, 0 elsewhere, bbar = 0; output: bbar on the leaves.  Every level runs as
// plain launches (no shared-memory tail).  Scratch over all cells: UST (the adjoint of u*
// on cells with children) and X, which holds G on level m-1 during a transposed
// restriction and ubar's other copy during a level's ping-pong sweeps.
template <class TV>
struct CycleT {
    ocg_hier* h;
    TV* U;
    TV* B;
    TV* X;
    TV* UST;
    TV* Tacc;
    Ctx& c;

    const HostTree& H() const { return h->t->H; }
    template <class F>
    void with_coefs(int m, F&& f) { Cycle<TV>{h, U, B, c}.with_coefs(m, f); }

    // ubar_K -= the accumulated B^m^T contributions (slots Tacc) for the coarser leaves K
    // (level m-1) of level m's T faces
    void gather(int m) {
        if (m < 1) return;
        const ocg_octree* t = h->t;
        const int k0 = t->tc_lo[m - 1], k1 = t->tc_hi[m - 1];
        if (k1 <= k0) return;
        launch(c, -1, m, k1 - k0, [&] {
            launch_k(kt_tgather<TV>, nblk(k1 - k0), BLK, 0, c.st, t->tables(), tree_levels(H()), t->level, t->tcoarse, k0,
                     k1, U, Tacc);
        });
        ck_launch("transposed gather");
    }
    // one transposed colour sweep from src to dst (U or X over level m); acc: add the
    // coarser leaves' shares to the slots Tacc
    void sweep(int m, int colour, TV* src, TV* dst, bool acc) {
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_SWEEP, m, A.ncell, [&] {
                launch_k(kt_fsweep<TV, TC, TW>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C,
                         (const TV*)src, dst, B, Tacc, colour, acc ? 1 : 0);
            });
        });
        ck_launch("transposed sweep");
    }
    // n pairs of transposed sweeps, colours (first, 1 - first) each; ubar ping-pongs
    // between U and X and ends in U (an even number of sweeps)
    void smooth(int m, int n, int first, bool acc) {
        TV* a = U;
        TV* b = X;
        for (int it = 0; it < n; ++it) {
            sweep(m, first, a, b, acc);
            sweep(m, 1 - first, b, a, acc);
        }
    }
    void coarsest(int m) {
        const int nu = h->prm.nu_coarsest, half = nu / 2;
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            const int nt = (int)std::min<int64_t>(256, (A.ncell / 8 + 31) / 32 * 32);
            launch(c, -1, m, A.ncell, [&] {
                launch_k(kt_coarsest<TV, TC, TW>, 1, nt, 0, c.st, A, h->t->tables(), C, U, B, X, nu - half, nu);
            });
        });
        ck_launch("transposed coarsest");
    }
    // transposes of the prolongation (before the recursion) and of the FAS restriction
    // and residual (after it) between levels m and m-1
    void prolong(int m) {
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_PROLONG, m, A.ncell, [&] {
                launch_k(kt_prolong<TV, TC, TW>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, UST);
            });
        });
        ck_launch("transposed prolong");
    }
    void restrict_(int m, bool acc) {
        const TV scale = TV(h->prm.beta_restrict / h->prm.alpha);
        const LevelArgs Ac = h->t->largs(m - 1);
        launch(c, OCG_PROBE_RESTRICT, m - 1, Ac.ncell, [&] {
            launch_k(kt_restrict_g<TV>, nblk(Ac.ncell), BLK, 0, c.st, Ac, h->t->tables(), U, B, UST, X);
        });
        with_coefs(m - 1, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            launch(c, OCG_PROBE_RESTRICT, m - 1, Ac.ncell, [&] {
                launch_k(kt_restrict_v<TV, TC, TW>, nblk(Ac.ncell / 8, OBLK), OBLK, 0, c.st, Ac, h->t->tables(), C, U, UST,
                         (const TV*)X);
            });
        });
        with_coefs(m, [&](auto C) {
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            const LevelArgs A = h->t->largs(m);
            launch(c, OCG_PROBE_RESTRICT, m, A.ncell, [&] {
                launch_k(kt_restrict_c<TV, TC, TW>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, h->t->tables(), C, U, B,
                         (const TV*)UST, (const TV*)X, Tacc, scale, acc ? 1 : 0);
            });
        });
        ck_launch("transposed restrict");
    }
    // last: no later visit of level m follows in this cycle, so what the steps after the
    // recursion would add to the coarser leaves (read only by a later visit of level m-1)
    // is not formed
    void cycle(int m, bool last) {
        if (m == H().mc) { coarsest(m); return; }
        smooth(m, h->prm.nu_post, 0, true);   // post-smoothing (colours 1, 0 per pair) transposed
        gather(m);
        prolong(m);
        const int mu = mu_at(h, m - 1);
        for (int k = 0; k < mu; ++k) cycle(m - 1, last && k == mu - 1);
        restrict_(m, !last);
        smooth(m, h->prm.nu_pre, 1, !last);   // pre-smoothing (colours 0, 1 per pair) transposed
        if (!last) gather(m);
    }
    // U, B: the leaf values of Z and zeros over the tree cells, zeros on the coarser levels
    template <class TZ>
    void seed(const TZ* Z) {
        const HostTree& HH = H();
        const int n = (int)HH.ntree;
        launch(c, -1, 0, n, [&] { launch_k(kt_seed<TV, TZ>, nblk(n), BLK, 0, c.st, n, h->t->flags, Z, U, B); });
        const int64_t rest = HH.ncell - HH.ntree;
        if (rest > 0) {
            ck(cudaMemsetAsync(U + HH.ntree, 0, rest * sizeof(TV), c.st), "memset");
            ck(cudaMemsetAsync(B + HH.ntree, 0, rest * sizeof(TV), c.st), "memset");
        }
    }
    void run() { cycle(H().D, true); }
};

void ensure_cycle_T(ocg_hier* h) {
    h->t->upload_adjoint();
    if (h->Xc) return;
    h->Xc = dalloc<double>(h->t->H.ncell);
    h->UST = dalloc<double>(h->t->H.ncell);
    const int64_t ns = std::max<int64_t>(6 * h->t->H.nt, 1);
    h->Tacc = dalloc<double>(ns);
    ck(cudaMemset(h->Tacc, 0, ns * sizeof(double)), "memset");
}

// ------------------------------------------------------------------ sweep autotuner
// For every level the cycle sweeps outside the shared-memory tail, capture 20 colour
// sweeps of each form into a graph, time 5 replays with CUDA events after 2 warm-up
// replays, and keep the faster form.  Sweeps act on the zeroed work vectors (b = 0 keeps
// u = 0), so tuning leaves no trace.
template <class TV>
void autotune_sweeps(ocg_hier* h) {
    const HostTree& H = h->t->H;
    if (!h->cap) ck(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t cs = h->cap;
    ck(cudaMemsetAsync(h->U, 0, cyc_len(H.ncell) * sizeof(double), cs), "memset");
    ck(cudaMemsetAsync(h->B, 0, cyc_len(H.ncell) * sizeof(double), cs), "memset");
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "cudaEventCreate");
    ck(cudaEventCreate(&e1), "cudaEventCreate");
    const int tail_top = h->tail_top[std::is_same<TV, double>::value ? 1 : 0];
    for (int m = H.D; m > H.mc; --m) {
        if (m <= tail_top && tail_top != TAIL_NONE) break;
        double us[4] = {0.0, 0.0, 0.0, 0.0};
        for (int form = 0; form < 4; ++form) {
            Ctx c{cs, nullptr, 0};
            Cycle<TV> cy{h, (TV*)h->U, (TV*)h->B, c};
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int q = 0; q < 20; ++q) cy.sweep(m, q & 1, 0, form);
            ck(cudaStreamEndCapture(cs, &g), "end capture");
            ck(cudaGraphInstantiate(&ge, g, 0), "graph instantiate");
            for (int w = 0; w < 2; ++w) ck(cudaGraphLaunch(ge, cs), "graph launch");
            ck(cudaEventRecord(e0, cs), "event");
            for (int r = 0; r < 5; ++r) ck(cudaGraphLaunch(ge, cs), "graph launch");
            ck(cudaEventRecord(e1, cs), "event");
            ck(cudaEventSynchronize(e1), "event sync");
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            us[form] = ms * 1000.0 / (5 * 20);
            cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
        }
        int best = OCG_SWEEP_OCTET;
        for (int form = 0; form < 4; ++form) {
            h->tune_us[m - H.mc][form] = us[form];
            if (us[form] < us[best]) best = form;
        }
        h->sweep_form[m - H.mc] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// ------------------------------------------------------------------ composite operator
// The device a hierarchy was set up on must be current for every call on it: its tables,
// coefficients and work vectors live in that device's memory.
void require_device(const ocg_hier* h) {
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != h->device)
        throw Status(OCG_EINVAL, "the hierarchy lives on device " + std::to_string(h->device) +
                                 ", the current device is " + std::to_string(dev));
}

int sm_count() {
    static int n[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) dev = 0;
    if (n[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        n[dev] = v;
    }
    return n[dev];
}

OMultiLevel tree_levels(const HostTree& H) {
    OMultiLevel ML{};
    ML.n = H.D + 1;
    int b = 0;
    for (int m = 0; m <= H.D; ++m) {
        ML.off[m] = (int)H.L(m).off;
        ML.noct[m] = (int)(H.L(m).ncell / 8);
        ML.ni[m] = H.L(m).ni;
        ML.boff[m] = b;
        b += (int)nblk(H.L(m).ncell / 8, OBLK);
    }
    ML.boff[H.D + 1] = b;
    return ML;
}

Red make_red(ocg_hier* h, int nb, int op, cudaGraphConditionalHandle cond = 0, int set_cond = 0) {
    Red R;
    R.part = h->part;
    R.cnt = h->cnt;
    R.S = h->S;
    R.nb = nb;
    R.op = op;
    R.nleaf = (double)h->t->H.nleaf;
    R.cond = cond;
    R.set_cond = set_cond;
    return R;
}

// Y = A P on the tree cells (P's inner entries are overwritten with child averages);
// op = OP_ALPHA also reduces (p, Ap) and forms alpha on the device.
template <class TO, class TC, class TW>
void apply_outer(ocg_hier* h, Coefs<TC, TW> C, TO* P, TO* Y, int op, Ctx& c) {
    const ocg_octree* t = h->t;
    const HostTree& H = t->H;
    for (int m = H.D; m >= 1; --m) {
        const LevelArgs A = t->largs(m);
        launch(c, -1, m, A.ncell, [&] {
            launch_k(k_oavg<TO, TC>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, t->tables(), C.d, P);
        });
    }
    ck_launch("avg");
    const OMultiLevel ML = tree_levels(H);
    // a bounded grid (blocks stride over the octet blocks): few partials to reduce
    const int nb = std::min(ML.boff[ML.n], 16 * sm_count());
    const Red R = make_red(h, nb, op);
    launch(c, OCG_PROBE_APPLY, 0, H.ntree, [&] {
        if constexpr (std::is_same<TO, double>::value && std::is_same<TC, float>::value) {
            const int nb2 = std::min(ML.boff[ML.n], 8 * sm_count());
            const Red R2 = make_red(h, nb2, op);
            launch_k(k_oapply_df2<VecD, OutD>, nb2, OBLK2, 0, c.st, ML, t->tables(), C, (const float*)h->rem32,
                     (const uint8_t*)t->flags, VecD{P}, OutD{Y}, R2);
        } else
            launch_k(k_oapply<TO, TC, TW>, nb, OBLK, 0, c.st, ML, t->tables(), C, P, Y, R);
    });
    ck_launch("apply");
}

// The mixed PCG's outer apply on p kept as FP32 pairs P = (ph, pl), the two halves of a
// tree-cell array (inner cells get the child means in pair form); Y in FP64.
void apply_outer_pp(ocg_hier* h, Coefs<float, float> C, float* ph, float* pl, double* Y, int op, Ctx& c) {
    const ocg_octree* t = h->t;
    const HostTree& H = t->H;
    for (int m = H.D; m >= 1; --m) {
        const LevelArgs A = t->largs(m);
        launch(c, -1, m, A.ncell, [&] {
            launch_k(k_oavg_pp<float>, nblk(A.ncell / 8, OBLK), OBLK, 0, c.st, A, t->tables(), C.d, ph, pl);
        });
    }
    ck_launch("avg");
    const OMultiLevel ML = tree_levels(H);
    const int nb = std::min(ML.boff[ML.n], 8 * sm_count());
    const Red R = make_red(h, nb, op);
    launch(c, OCG_PROBE_APPLY, 0, H.ntree, [&] {
        launch_k(k_oapply_df2<VecP, OutD>, nb, OBLK2, 0, c.st, ML, t->tables(), C, (const float*)h->rem32,
                 (const uint8_t*)t->flags, VecP{ph, pl}, OutD{Y}, R);
    });
    ck_launch("apply");
}

// Y = A^T P on the leaves: A P, then the A^T - A rows around the T-junctions.
// op: the reduction fused into the forward part, over (p, A p) = (p, A^T p).
template <class TO, class TC, class TW>
void apply_outer_T(ocg_hier* h, Coefs<TC, TW> C, TO* P, TO* Y, Ctx& c, int op = OP_NONE) {
    const ocg_octree* t = h->t;
    apply_outer<TO, TC, TW>(h, C, P, Y, op, c);
    const HostTree& H = t->H;
    if (H.nt == 0) return;
    const Tables T = t->tables();
    launch(c, -1, 0, H.nt, [&] {
        launch_k(k_tfine<TO, TC, TW>, nblk(H.nt, OBLK), OBLK, 0, c.st, T, C, t->t_oct, P, Y, h->tseed);
    });
    launch(c, -1, 0, t->n_tcoarse, [&] {
        launch_k(k_tcoarse<TO, TC, TW>, nblk(t->n_tcoarse), BLK, 0, c.st, T, C, tree_levels(H), t->level, t->tcoarse,
                                                                    t->n_tcoarse, P, Y);
    });
    launch(c, -1, 0, t->n_tdesc, [&] {
        launch_k(k_tdesc<TO>, nblk(t->n_tdesc), BLK, 0, c.st, T, t->tdesc, t->n_tdesc, (int)H.ntree, t->flags, h->tseed, Y);
    });
    ck_launch("apply_T correction");
}

// ------------------------------------------------------------------ PCG (Alg. 1)
// The loop is split so that a WHILE body holds exactly one iteration:
//   begin:  r = b; ||b|| (null-space shift); z = M r; rho = (r, z); p = z; half_a
//   body:   half_b; half_a                    (repeated while not converged)
//   half_a: Ap = A p, alpha; x += alpha p, r -= alpha Ap; ||r|| test (sets the condition)
//   half_b: z = M r; beta; p = z + beta p
//   finish: true residual ||b - A x|| in FP64
// S[S_XMEAN] = mean of the solution over the leaves (xt holds it in FP64; inner cells 0).
// The averaging pass of the true-residual apply wrote child means into xt's inner cells,
// so the sum runs over leaves through the flags.
void solution_mean(ocg_hier* h, Ctx& c, const double* xt) {
    const int n = (int)h->t->H.ntree;
    const unsigned rb = std::min<unsigned>(nblk(n), (unsigned)h->red_blocks);
    launch(c, -1, 0, n, [&] {
        launch_k(k_leafsum, rb, BLK, 0, c.st, xt, h->t->flags, n, make_red(h, rb, OP_XMEAN));
    });
}

template <class TO, class TV, class TC, class TW, bool TR>
struct PcgImpl {
    ocg_hier* h;
    Coefs<TC, TW> Co;
    bool ns;
    Ctx& c;
    cudaGraphConditionalHandle cond;
    int set_cond;
    bool warm = false;   // x0 from xt (OCG_SOLVE_WARM) instead of 0

    const HostTree& H() const { return h->t->H; }
    TO* x() { return (TO*)h->x; }
    TO* r() { return (TO*)h->r; }
    TO* p() { return (TO*)h->p; }
    TO* Ap() { return (TO*)h->Ap; }
    TV* U() { return (TV*)h->U; }
    TV* B() { return (TV*)h->B; }
    int n() const { return (int)H().ntree; }
    unsigned gb() const { return nblk(H().ntree); }
    unsigned rb() const { return std::min<unsigned>(nblk(H().ntree), (unsigned)h->red_blocks); }
    void zero(void* ptr, size_t bytes) { ck(cudaMemsetAsync(ptr, 0, bytes, c.st), "memset"); }
    // the mixed forward solve keeps p as FP32 pairs: hi in the first n floats of the FP64
    // array, lo in the next n
    static constexpr bool PP = !TR && std::is_same<TO, double>::value && std::is_same<TC, float>::value;
    // the forward cycle keeps u and b in the cycle layout (cyc); the transposed one does not
    static constexpr bool CY = !TR;
    float* hi(double* v) { return (float*)v; }
    float* lo(double* v) { return (float*)v + n(); }
    void pupdate(int first) {
        launch(c, -1, 0, n(), [&] {
            if constexpr (PP)
                launch_k(k_pupdate_pp<TV>, gb(), BLK, 0, c.st, hi(h->p), lo(h->p), (const TV*)Z(), (const double*)h->S,
                         n(), first);
            else
                launch_k(k_pupdate<TO, TV, CY>, gb(), BLK, 0, c.st, p(), Z(), h->S, n(), first);
        });
    }

    void begin() {
        if (warm) launch(c, -1, 0, n(), [&] { launch_k(k_cast<double, TO>, gb(), BLK, 0, c.st, h->xt, x(), n()); });
        else zero(h->x, n() * sizeof(TO));
        zero(h->p, n() * sizeof(TO));
        zero(h->B, cyc_len(H().ncell) * sizeof(TV));
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<double, TO>, gb(), BLK, 0, c.st, h->bt, r(), n()); });
        launch(c, -1, 0, n(), [&] { launch_k(k_dot<TO, TO, true>, rb(), BLK, 0, c.st, r(), r(), n(), make_red(h, rb(), OP_BB)); });
        if (warm) {
            // r = b - A x0 (A^T x0); ||b|| above stays the reference of the stop test
            if constexpr (TR) apply_outer_T<TO, TC, TW>(h, Co, x(), Ap(), c);
            else apply_outer<TO, TC, TW>(h, Co, x(), Ap(), OP_NONE, c);
            launch(c, -1, 0, n(), [&] { launch_k(k_sub<TO>, gb(), BLK, 0, c.st, r(), (const TO*)Ap(), n()); });
        }
        // (the mixed solve forms the first cycle's first sweep here, as in the Krylov update)
        const FirstSweep F = first_sweep_args();
        launch(c, -1, 0, n(), [&] { launch_k(k_project<TO, TV, CY>, gb(), BLK, 0, c.st, r(), h->t->flags, h->S, B(), n(), F); });
        ck_launch("begin");
        first_done = F.u32 != nullptr;
        precondition();
        launch(c, -1, 0, n(), [&] { launch_k(k_dot<TO, TV, false, CY>, rb(), BLK, 0, c.st, r(), Z(), n(), make_red(h, rb(), OP_RZ0)); });
        pupdate(1);
        ck_launch("begin");
        half_a();
    }
    // z = M r (forward: r in B, z in U) or z = M^T r (transpose: r in B, z in B)
    TV* Z() { return TR ? B() : U(); }
    // the Krylov update forms the next cycle's first sweep (FirstSweep); first_done: the
    // preceding half iteration did (a loop body always follows one)
    bool fuse_first() const {
        if constexpr (!TR && std::is_same<TV, float>::value) return first_sweep_fusable(h);
        else return false;
    }
    bool first_done = false;
    FirstSweep first_sweep_args() const {
        if (!fuse_first()) return FirstSweep{nullptr, nullptr, 0, 0};
        const LevelArgs AD = h->t->largs(H().D);
        return FirstSweep{(float*)h->U, h->c32[0], AD.off, AD.off + AD.ncell};
    }
    void precondition() {
        if constexpr (TR) {
            CycleT<TV> ct{h, U(), B(), (TV*)h->Xc, (TV*)h->UST, (TV*)h->Tacc, c};
            ct.seed((const TV*)B());
            ct.run();
        } else {
            Cycle<TV> cy{h, U(), B(), c};
            if (first_done) cy.skip_first = true;
            else zero(h->U, cyc_len(H().ntree) * sizeof(TV));   // the tree cells' positions and a few coarse cells
            first_done = false;
            cy.run();
        }
    }
    void half_a() {
        if constexpr (TR) apply_outer_T<TO, TC, TW>(h, Co, p(), Ap(), c, OP_ALPHA);
        else if constexpr (PP) apply_outer_pp(h, Co, hi(h->p), lo(h->p), h->Ap, OP_ALPHA, c);
        else apply_outer<TO, TC, TW>(h, Co, p(), Ap(), OP_ALPHA, c);
        launch(c, -1, 0, n(), [&] {
            const Red R = make_red(h, rb(), OP_RR, cond, set_cond);
            if constexpr (PP) {
                const FirstSweep F = first_sweep_args();
                if (ns)
                    launch_k(k_update_pp<true>, rb(), BLK, 0, c.st, h->x, h->r, (const float*)hi(h->p),
                             (const float*)lo(h->p), (const double*)h->Ap, (const uint8_t*)h->t->flags,
                             (float*)B(), n(), R, F);
                else
                    launch_k(k_update_pp<false>, rb(), BLK, 0, c.st, h->x, h->r, (const float*)hi(h->p),
                             (const float*)lo(h->p), (const double*)h->Ap, (const uint8_t*)nullptr,
                             (float*)B(), n(), R, F);
            } else {
                // under the null space k_project below writes b (and the first sweep)
                if (ns) launch_k(k_update<TO, TV, true, CY>, rb(), BLK, 0, c.st, x(), r(), p(), Ap(), nullptr, n(), R,
                                 FirstSweep{});
                else launch_k(k_update<TO, TV, false, CY>, rb(), BLK, 0, c.st, x(), r(), p(), Ap(), B(), n(), R,
                              first_sweep_args());
            }
        });
        // the zero-mean shift of r (fused into the update of the pair-stored mixed form)
        if (ns && !PP)
            launch(c, -1, 0, n(), [&] {
                launch_k(k_project<TO, TV, CY>, gb(), BLK, 0, c.st, r(), h->t->flags, h->S, B(), n(), first_sweep_args());
            });
        ck_launch("half_a");
    }
    void half_b() {
        precondition();
        launch(c, -1, 0, n(), [&] { launch_k(k_dot<TO, TV, false, CY>, rb(), BLK, 0, c.st, r(), Z(), n(), make_red(h, rb(), OP_BETA)); });
        pupdate(0);
        ck_launch("half_b");
    }
    void body() {
        first_done = fuse_first();
        half_b();
        half_a();
    }
    void finish() {
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<TO, double>, gb(), BLK, 0, c.st, x(), h->xt, n()); });
        if constexpr (TR) apply_outer_T<double, TC, TW>(h, Co, h->xt, h->yt, c);
        else apply_outer<double, TC, TW>(h, Co, h->xt, h->yt, OP_NONE, c);
        launch(c, -1, 0, n(), [&] {
            launch_k(k_resid<double>, rb(), BLK, 0, c.st, h->bt, h->yt, h->t->flags, n(), make_red(h, rb(), OP_TRUE));
        });
        if (ns) solution_mean(h, c, h->xt);
        ck_launch("finish");
    }
};

// Alg. 1 on A x = b, and Alg. 1 on the adjoint system A^T x = b preconditioned by the
// transposed cycle M^T (no counterpart in the paper): its scalars (r, M^T r) = (M r, r) and
// (p, A^T p) = (A p, p) are the forward method's quadratic forms.
template <class TO, class TV, class TC, class TW>
using Pcg = PcgImpl<TO, TV, TC, TW, false>;
template <class TO, class TV, class TC, class TW>
using PcgT = PcgImpl<TO, TV, TC, TW, true>;

// ------------------------------------------------------- BiCGStab (adjoint system)
// Solves A^T x = b, right-preconditioned by the same mu-cycle (the cycle approximates
// A^{-1}; Alg. 1 with it stagnates on A^T because A is not symmetric at T-junctions).
//   begin: r = rhat = b (null-space shift), rho = (rhat, r), condition
//   body:  p = r + beta (p - omega v); ph = M p; v = A^T ph; alpha = rho / (rhat, v);
//          s = r - alpha v; sh = M s; t = A^T sh; omega = (t, s) / (t, t);
//          x += alpha ph + omega sh; r = s - omega t; ||r|| test, rho, beta
//   finish: true residual ||b - A^T x|| in FP64
template <class TO, class TV, class TC, class TW>
struct BiCG {
    ocg_hier* h;
    Coefs<TC, TW> Co;
    bool ns;
    Ctx& c;
    cudaGraphConditionalHandle cond;
    int set_cond;
    bool warm = false;   // x0 from xt (OCG_SOLVE_WARM) instead of 0

    const HostTree& H() const { return h->t->H; }
    TO* V(double* p) { return (TO*)p; }
    TV* U() { return (TV*)h->U; }
    TV* B() { return (TV*)h->B; }
    int n() const { return (int)H().ntree; }
    unsigned gb() const { return nblk(H().ntree); }
    unsigned rb() const { return std::min<unsigned>(nblk(H().ntree), (unsigned)h->red_blocks); }
    void zero(void* ptr, size_t bytes) { ck(cudaMemsetAsync(ptr, 0, bytes, c.st), "memset"); }

    void begin() {
        if (warm) launch(c, -1, 0, n(), [&] { launch_k(k_cast<double, TO>, gb(), BLK, 0, c.st, h->xt, V(h->x), n()); });
        else zero(h->x, n() * sizeof(TO));
        zero(h->p, n() * sizeof(TO));
        zero(h->B, H().ncell * sizeof(TV));
        TO* r = V(h->r);
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<double, TO>, gb(), BLK, 0, c.st, h->bt, r, n()); });
        launch(c, -1, 0, n(), [&] { launch_k(k_dot<TO, TO, true>, rb(), BLK, 0, c.st, r, r, n(), make_red(h, rb(), OP_BB)); });
        if (warm) {
            // r = b - A^T x0; ||b|| above stays the reference of the stop test
            apply_outer_T<TO, TC, TW>(h, Co, V(h->x), V(h->Ap), c);
            launch(c, -1, 0, n(), [&] { launch_k(k_sub<TO>, gb(), BLK, 0, c.st, r, (const TO*)V(h->Ap), n()); });
        }
        zero(h->Ap, n() * sizeof(TO));
        if (ns)
            launch(c, -1, 0, n(), [&] {
                launch_k(k_project<TO, TV>, gb(), BLK, 0, c.st, r, h->t->flags, h->S, (TV*)nullptr, n(), FirstSweep{});
            });
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<TO, TO>, gb(), BLK, 0, c.st, r, V(h->rhat), n()); });
        launch(c, -1, 0, n(), [&] {
            launch_k(k_dot<TO, TO, false>, rb(), BLK, 0, c.st, V(h->rhat), r, n(), make_red(h, rb(), OP_BI_INIT, cond, set_cond));
        });
        ck_launch("bicg begin");
    }
    // out = M^T (the value that k_bi_p / k_bi_s left in B)
    void precondition(TO* out) {
        CycleT<TV> ct{h, U(), B(), (TV*)h->Xc, (TV*)h->UST, (TV*)h->Tacc, c};
        ct.seed((const TV*)B());
        ct.run();
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<TV, TO>, gb(), BLK, 0, c.st, B(), out, n()); });
    }
    void body() {
        TO *r = V(h->r), *p = V(h->p), *v = V(h->Ap), *s = V(h->s), *t = V(h->tv), *ph = V(h->ph), *sh = V(h->sh);
        launch(c, -1, 0, n(), [&] { launch_k(k_bi_p<TO, TV>, gb(), BLK, 0, c.st, p, r, v, B(), h->S, n()); });
        precondition(ph);
        apply_outer_T<TO, TC, TW>(h, Co, ph, v, c);
        launch(c, -1, 0, n(), [&] {
            launch_k(k_dot<TO, TO, false>, rb(), BLK, 0, c.st, V(h->rhat), v, n(), make_red(h, rb(), OP_BI_ALPHA));
        });
        launch(c, -1, 0, n(), [&] { launch_k(k_bi_s<TO, TV>, gb(), BLK, 0, c.st, s, r, v, B(), h->S, n()); });
        precondition(sh);
        apply_outer_T<TO, TC, TW>(h, Co, sh, t, c);
        launch(c, -1, 0, n(), [&] { launch_k(k_dot2<TO>, rb(), BLK, 0, c.st, t, s, n(), make_red(h, rb(), OP_BI_OMEGA)); });
        launch(c, -1, 0, n(), [&] {
            launch_k(k_bi_x<TO>, rb(), BLK, 0, c.st, V(h->x), r, s, t, ph, sh, V(h->rhat), n(),
                                               make_red(h, rb(), OP_BI_RR, cond, set_cond));
        });
        if (ns)
            launch(c, -1, 0, n(), [&] {
                launch_k(k_project<TO, TV>, gb(), BLK, 0, c.st, r, h->t->flags, h->S, (TV*)nullptr, n(), FirstSweep{});
            });
        ck_launch("bicg body");
    }
    void finish() {
        launch(c, -1, 0, n(), [&] { launch_k(k_cast<TO, double>, gb(), BLK, 0, c.st, V(h->x), h->xt, n()); });
        apply_outer_T<double, TC, TW>(h, Co, h->xt, h->yt, c);
        launch(c, -1, 0, n(), [&] {
            launch_k(k_resid<double>, rb(), BLK, 0, c.st, h->bt, h->yt, h->t->flags, n(), make_red(h, rb(), OP_TRUE));
        });
        if (ns) solution_mean(h, c, h->xt);
        ck_launch("bicg finish");
    }
};

// Capture begin; WHILE(not converged) { body }; finish into one graph.  Solver is Pcg or
// BiCG (both: begin / body / finish, the reduction that ends each of begin and body sets
// the WHILE condition).
template <template <class, class, class, class> class Solver, class TO, class TV, class TC, class TW>
void build_graph(ocg_hier* h, Coefs<TC, TW> Co, bool ns, bool warm, GraphSolve& gs) {
    if (!h->cap) ck(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t cs = h->cap;
    Ctx c{cs, nullptr, 0};
    ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus stt;
    try {
        ck(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
        cudaGraphConditionalHandle cond;
        ck(cudaGraphConditionalHandleCreate(&cond, g, 0, 0), "conditional handle");
        Solver<TO, TV, TC, TW> pc{h, Co, ns, c, cond, 1};
        pc.warm = warm;
        pc.begin();
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        ck(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, &deps, nullptr, &ndeps), "capture info");
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode;
        ck(cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, &np), "add WHILE node");
        cudaGraph_t body = np.conditional.phGraph_out[0];
        ck(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies),
           "update capture dependencies");
        const int64_t before_finish = c.count;
        pc.finish();
        gs.outer_kernels = c.count;
        (void)before_finish;
        ck(cudaStreamEndCapture(cs, &g), "end capture");
        // the body: one iteration, captured into the WHILE node's child graph
        Ctx cb{cs, nullptr, 0};
        ck(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
           "begin body capture");
        Solver<TO, TV, TC, TW> pb{h, Co, ns, cb, cond, 1};
        pb.warm = warm;
        pb.body();
        cudaGraph_t bg = nullptr;
        ck(cudaStreamEndCapture(cs, &bg), "end body capture");
        gs.body_kernels = cb.count;
        ck(cudaGraphInstantiate(&gs.exec, g, 0), "graph instantiate");
        gs.graph = g;
    } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        if (junk) cudaGraphDestroy(junk);
        cudaGetLastError();
        throw;
    }
}

void ensure_work(ocg_hier* h) {
    if (h->S) return;
    const HostTree& H = h->t->H;
    const int64_t n = H.ntree;
    for (double** v : {&h->x, &h->r, &h->p, &h->Ap, &h->bt, &h->xt, &h->yt}) *v = dalloc<double>(n);
    // the cycle's u and b: FP64 or FP32, in the cycle layout (whole 64-cell groups)
    h->U = dalloc<double>(cyc_len(H.ncell));
    h->B = dalloc<double>(cyc_len(H.ncell));
    h->S = dalloc<double>(S_COUNT);
    ck(cudaMallocHost((void**)&h->hS, S_COUNT * sizeof(double)), "cudaMallocHost");
    h->part = dalloc<double>(3 * ((int64_t)nblk(n) + H.D + 8));
    h->cnt = dalloc<unsigned>(1);
    ck(cudaMemset(h->cnt, 0, sizeof(unsigned)), "memset");
    ck(cudaMemset(h->S, 0, S_COUNT * sizeof(double)), "memset");
}

void ensure_adjoint(ocg_hier* h) {
    h->t->upload_adjoint();
    if (h->tseed) return;
    h->tseed = dalloc<double>(h->t->H.ntree);
    ck(cudaMemset(h->tseed, 0, h->t->H.ntree * sizeof(double)), "memset");
}

void ensure_bicg(ocg_hier* h) {
    ensure_adjoint(h);
    ensure_cycle_T(h);
    if (h->rhat) return;
    const int64_t n = h->t->H.ntree;
    for (double** v : {&h->rhat, &h->s, &h->tv, &h->ph, &h->sh}) *v = dalloc<double>(n);
}

template <template <class, class, class, class> class Solver, class TO, class TV, class TC, class TW>
int krylov_solve(ocg_hier* h, Coefs<TC, TW> Co, int prec, const double* b_user, double* x_user,
                 const ocg_solve_params* sp, ocg_solve_stats* stats, cudaStream_t st) {
    const ocg_octree* t = h->t;
    const HostTree& H = t->H;
    const bool transpose = (sp->flags & OCG_SOLVE_TRANSPOSE) != 0;
    const bool bicg = transpose && (sp->flags & OCG_SOLVE_BICGSTAB) != 0;
    const bool warm = (sp->flags & OCG_SOLVE_WARM) != 0;
    const bool ns = sp->nullspace < 0 ? h->ns_auto : sp->nullspace != 0;
    const bool eager = (sp->flags & OCG_SOLVE_EAGER) || h->probe.kind != OCG_PROBE_OFF;
    // scalars: tolerance, iteration cap, null-space flag, counters
    std::memset(h->hS, 0, S_COUNT * sizeof(double));
    h->hS[S_NS] = ns ? 1.0 : 0.0;
    h->hS[S_TOL] = sp->tol;
    h->hS[S_MAXIT] = sp->max_iter;
    Ctx c{st, &h->probe, 0};
    ck(cudaMemcpyAsync(h->S, h->hS, S_COUNT * sizeof(double), cudaMemcpyHostToDevice, st), "copy scalars");
    ck(cudaMemsetAsync(h->bt, 0, H.ntree * sizeof(double), st), "memset");
    launch(c, -1, 0, H.nleaf, [&] {
        launch_k(k_scatter<double, double>, nblk(H.nleaf), BLK, 0, st, b_user, h->bt, t->leaf_cell, (int)H.nleaf);
    });
    if (warm) {
        // the initial guess, on the leaves of the FP64 tree vector (begin casts it to x)
        ck(cudaMemsetAsync(h->xt, 0, H.ntree * sizeof(double), st), "memset");
        launch(c, -1, 0, H.nleaf, [&] {
            launch_k(k_scatter<double, double>, nblk(H.nleaf), BLK, 0, st, (const double*)x_user, h->xt, t->leaf_cell,
                     (int)H.nleaf);
        });
    }
    ck_launch("scatter");
    int64_t kernels = c.count;
    GraphSolve& gs = h->graphs[!transpose ? 0 : (bicg ? 2 : 1)][prec][ns ? 1 : 0][warm ? 1 : 0];
    const bool unrolled = (sp->flags & OCG_SOLVE_UNROLLED) != 0;
    if (unrolled) {
        // measurement form: exactly max_iter iterations captured into one flat graph (no
        // WHILE node), so probe events become event-record nodes between the kernels
        if (!h->cap) ck(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
        Ctx cc{h->cap, &h->probe, 0};
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        ck(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            Solver<TO, TV, TC, TW> pc{h, Co, ns, cc, 0, 0};
            pc.warm = warm;
            pc.begin();
            const int nbody = bicg ? sp->max_iter : sp->max_iter - 1;
            for (int q = 0; q < nbody; ++q) pc.body();
            pc.finish();
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(h->cap, &junk);
            if (junk) cudaGraphDestroy(junk);
            cudaGetLastError();
            throw;
        }
        ck(cudaStreamEndCapture(h->cap, &g), "end capture");
        ck(cudaGraphInstantiate(&ge, g, 0), "graph instantiate");
        ck(cudaGraphLaunch(ge, st), "graph launch");
        ck(cudaStreamSynchronize(st), "stream sync");
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        kernels = cc.count;
    } else if (eager) {
        Solver<TO, TV, TC, TW> pc{h, Co, ns, c, 0, 0};
        pc.warm = warm;
        pc.begin();
        while (true) {
            ck(cudaMemcpyAsync(h->hS, h->S, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st), "copy scalars");
            ck(cudaStreamSynchronize(st), "stream sync");
            if (h->hS[S_DONE] != 0.0) break;
            pc.body();
        }
        pc.finish();
        kernels = c.count;
    } else {
        if (!gs.exec) build_graph<Solver, TO, TV, TC, TW>(h, Co, ns, warm, gs);
        ck(cudaGraphLaunch(gs.exec, st), "graph launch");
    }
    // the solution is read from xt (FP64 copy of x made by finish), shifted to zero mean
    // under the null space
    launch(c, -1, 0, H.nleaf, [&] {
        if (ns)
            launch_k(k_gather_shift<double, double>, nblk(H.nleaf), BLK, 0, st, h->xt, x_user, t->leaf_cell, h->S,
                                                                         (int)H.nleaf);
        else
            launch_k(k_gather<double, double>, nblk(H.nleaf), BLK, 0, st, h->xt, x_user, t->leaf_cell, (int)H.nleaf);
    });
    ck_launch("gather");
    ck(cudaMemcpyAsync(h->hS, h->S, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st), "copy scalars");
    ck(cudaStreamSynchronize(st), "stream sync");
    const double* S = h->hS;
    const int k = (int)S[S_K];
    if (unrolled) {
        kernels += c.count;   // captured kernels + scatter and gather
    } else if (!eager) {
        // PCG's begin ends with the first half iteration, so its WHILE body runs k - 1
        // times; BiCGStab's body runs k times
        const int64_t body_runs = bicg ? k : std::max(k - 1, 0);
        kernels = c.count + gs.outer_kernels + body_runs * gs.body_kernels;
    } else {
        kernels = c.count;
    }
    g_launches += kernels;
    std::memset(stats, 0, sizeof(*stats));
    const double bb = S[S_BB];
    stats->iterations = k;
    stats->hist[0] = 1.0;
    for (int q = 1; q <= k && q < OCG_HIST; ++q) stats->hist[q] = S[S_HIST + q];
    stats->rel_res = bb > 0.0 ? std::sqrt(std::max(S[S_RR], 0.0) / bb) : 0.0;
    stats->true_rel_res = bb > 0.0 ? std::sqrt(std::max(S[S_TRUE], 0.0) / bb) : 0.0;
    stats->kernels = kernels;
    const bool conv = !(stats->rel_res > sp->tol);
    stats->converged = conv ? 1 : 0;
    if (!std::isfinite(stats->rel_res) || !std::isfinite(stats->true_rel_res)) {
        g_err = "non-finite residual norm";
        return OCG_ENAN;
    }
    if (!conv) {
        g_err = "Krylov loop reached max_iter before the tolerance";
        return OCG_ENOTCONV;
    }
    return OCG_OK;
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

int ocg_octree_rebuild(const ocg_octree* prev, const ocg_octree_desc* desc, const double box[6], ocg_octree** out) {
    return guard([&] {
        if (!prev || !desc || !box || !out) throw Status(OCG_EINVAL, "null argument");
        *out = nullptr;
        std::unique_ptr<ocg_octree> t(new ocg_octree());
        try {
            rebuild_host_tree(prev->H, *desc, box, t->H);
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
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < H.nleaf; ++r)
            for (int dir = 0; dir < 6; ++dir) {
                int8_t kd;
                int64_t rk;
                leaf_neighbour(H, r, dir, kd, rk);
                if (kind) kind[6 * r + dir] = kd;
                if (rank) rank[6 * r + dir] = rk;
            }
    });
}

int ocg_octree_export_faces(const ocg_octree* t, int32_t* axis, int32_t* depth, int32_t* i, int32_t* j,
                            int32_t* k, int64_t* minus, int64_t* plus) {
    return guard([&] {
        if (!t) throw Status(OCG_EINVAL, "null octree");
        const HostTree& H = t->H;
        export_faces(H, 0, H.nface, axis, depth, i, j, k, minus, plus);
    });
}

int ocg_octree_export_faces_range(const ocg_octree* t, int64_t first, int64_t count, int32_t* axis,
                                  int32_t* depth, int32_t* i, int32_t* j, int32_t* k, int64_t* minus,
                                  int64_t* plus) {
    return guard([&] {
        if (!t) throw Status(OCG_EINVAL, "null octree");
        const HostTree& H = t->H;
        if (first < 0 || count < 0 || first + count > H.nface) throw Status(OCG_EINVAL, "face range");
        export_faces(H, first, count, axis, depth, i, j, k, minus, plus);
    });
}

int ocg_octree_export_level(const ocg_octree* t, int32_t m, int64_t* n, int32_t* i, int32_t* j, int32_t* k,
                            int8_t* leaf) {
    return guard([&] {
        if (!t || !n) throw Status(OCG_EINVAL, "null argument");
        const HostTree& H = t->H;
        if (m < H.mc || m > H.D) throw Status(OCG_EINVAL, "level out of range");
        const std::vector<int64_t> cells = level_cells_morton(H, m);
        if (i) {
            for (size_t c = 0; c < cells.size(); ++c) {
                int64_t a, b, d;
                H.cell_coords(m, cells[c], a, b, d);
                i[c] = (int32_t)a; j[c] = (int32_t)b; k[c] = (int32_t)d;
                if (leaf) leaf[c] = (int8_t)(H.cell_flags[cells[c]] & 1);
            }
        }
        *n = (int64_t)cells.size();
    });
}

// Geometric multigrid (ablation of Sec. 3.3): every cell with children on the levels below
// the finest gets the coefficients of the grid at its own size H (ocg_mg_params.coarsening),
// computed on the host from the description's solids and written over Alg. 3's FP64 set.
void rediscretise(ocg_hier* h, cudaStream_t st) {
    const HostTree& H = h->t->H;
    std::vector<int64_t> idx;
    std::vector<double> vd, vc[3];
    for (int m = H.D - 1; m >= H.mc; --m) {
        const LevelMeta& l = H.L(m);
        const double hm = 1.0 / ((double)H.n0 * std::ldexp(1.0, m));
        const int64_t N = l.N;
        const size_t base = idx.size();
        std::vector<int64_t> cells;
        for (int64_t g = l.off; g < l.off + l.ncell; ++g)
            if (H.child_oct[g] >= 0 && (H.cell_flags[g] & 2)) cells.push_back(g);
        idx.resize(base + cells.size());
        vd.resize(idx.size());
        for (auto& v : vc) v.resize(idx.size());
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < (int64_t)cells.size(); ++q) {
            const int64_t g = cells[q];
            int64_t c[3];
            H.cell_coords(m, g, c[0], c[1], c[2]);
            double total = 0.0;
            for (int a = 0; a < 3; ++a) {
                for (int side = 0; side < 2; ++side) {
                    int64_t p[3] = {c[0], c[1], c[2]};
                    p[a] += side;                        // the + face is the - face of (c + e_a)
                    const bool wall = side == 0 ? p[a] - 1 < 0 : p[a] >= N;
                    const double w = wall ? (h->bc[2 * a + side] == OCG_BC_DIRICHLET ? 2.0 * hm : 0.0)
                                          : (double)face_beta_geometric(H.desc, m, a, p[0], p[1], p[2]) * hm;
                    total += w;
                    if (side == 0) vc[a][base + q] = -w;
                }
            }
            idx[base + q] = g;
            vd[base + q] = total;
        }
    }
    const int64_t n = (int64_t)idx.size();
    if (n == 0) return;
    int64_t* didx = dupload(idx);
    double* dv[4] = {dupload(vd), dupload(vc[0]), dupload(vc[1]), dupload(vc[2])};
    launch_k(k_set_coefs, nblk(n), BLK, 0, st, (int)n, (const int64_t*)didx, (const double*)dv[0],
             (const double*)dv[1], (const double*)dv[2], (const double*)dv[3], h->c64[0], h->c64[1], h->c64[2],
             h->c64[3]);
    ck_launch("rediscretise");
    ck(cudaStreamSynchronize(st), "setup sync");
    dfree(didx);
    for (double* v : dv) dfree(v);
}

// The coefficient sets of a hierarchy from the face fractions beta (canonical face order):
// the face scatter and leaf gather (Sec. 3.1), Alg. 3 on every level (or the geometric
// rediscretisation), the FP32 / BF16 copies.  Arrays are allocated on first use and
// rewritten in place afterwards, so graphs captured on the hierarchy stay valid.
void build_coefficients(ocg_hier* h, const float* beta, cudaStream_t st) {
    const ocg_octree* t = h->t;
    const HostTree& H = t->H;
    const int64_t ntw = 24 * std::max<int64_t>(H.nt, 1);
    if (!h->c64[0]) h->c64[0] = dalloc<double>(H.ncell);
    if (!h->tw64) h->tw64 = dalloc<double>(ntw);
    double* cm = dalloc<double>(3 * H.ncell);   // c_x-, c_y-, c_z- as one [3][ncell] block
    ck(cudaMemsetAsync(h->c64[0], 0, H.ncell * sizeof(double), st), "memset");
    ck(cudaMemsetAsync(cm, 0, 3 * H.ncell * sizeof(double), st), "memset");
    ck(cudaMemsetAsync(h->tw64, 0, ntw * sizeof(double), st), "memset");
    std::vector<double> hd(H.D + 1);
    for (int d = 0; d <= H.D; ++d) hd[d] = 1.0 / (double)((int64_t)H.n0 << d);
    double* dh = dupload(hd);
    int* derr = dalloc<int>(1);
    ck(cudaMemsetAsync(derr, 0, sizeof(int), st), "memset");
    if (H.nface > 0) {
        launch_k(k_face_scatter, nblk(H.nface), BLK, 0, st, beta, t->fslot, t->fkind, t->fdepth, dh, (int)H.nface, cm,
                                                     h->tw64, derr);
        ck_launch("face scatter");
    }
    LevelTab LT{};
    LT.mc = H.mc;
    for (int m = H.mc; m <= H.D; ++m) {
        LT.off[m - H.mc] = (int)H.L(m).off;
        LT.h[m - H.mc] = H.L(m).h;
    }
    launch_k(k_leaf_gather, nblk(H.nleaf), BLK, 0, st, t->leaf_cell, t->level, t->tables(), LT,
                                                make_int4(h->bc[0], h->bc[1], h->bc[2], h->bc[3]), make_int2(h->bc[4], h->bc[5]),
                                                (int)H.nleaf, (int)H.ncell, h->c64[0], cm, h->tw64);
    ck_launch("leaf gather");
    for (int m = H.D; m > H.mc; --m) {
        const LevelArgs A = t->largs(m);
        launch_k(k_coarsen, nblk(A.ncell / 8), BLK, 0, st, A, t->tables(), h->prm.alpha, h->c64[0], cm, (int)H.ncell);
        ck_launch("coarsen");
    }
    for (int q = 0; q < 3; ++q) {
        if (!h->c64[q + 1]) h->c64[q + 1] = dalloc<double>(H.ncell);
        ck(cudaMemcpyAsync(h->c64[q + 1], cm + q * H.ncell, H.ncell * sizeof(double), cudaMemcpyDeviceToDevice, st),
           "copy");
    }
    int herr = 0;
    ck(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "setup sync");
    dfree(cm); dfree(dh); dfree(derr);
    if (herr) throw Status(OCG_EINVAL, "face beta must be finite and >= 0");
    if (h->prm.coarsening == OCG_COARSEN_GEOMETRIC) rediscretise(h, st);
    if (h->prm.coef_dtype == OCG_F32) {
        for (int q = 0; q < 4; ++q) {
            if (!h->c32[q]) h->c32[q] = dalloc<float>(H.ncell);
            launch_k(k_convert<float>, nblk(H.ncell), BLK, 0, st, h->c64[q], h->c32[q], H.ncell);
            if (h->prm.bf16_coarse && q > 0) {
                if (!h->c16[q]) h->c16[q] = dalloc<__nv_bfloat16>(H.ncell);
                launch_k(k_convert<__nv_bfloat16>, nblk(H.ncell), BLK, 0, st, h->c64[q], h->c16[q], H.ncell);
            }
        }
        if (!h->tw32) h->tw32 = dalloc<float>(ntw);
        launch_k(k_convert<float>, nblk(ntw), BLK, 0, st, h->tw64, h->tw32, ntw);
        // the outer apply's diagonal remainder, from the FP64 diagonal and the stored FP32 faces
        if (!h->rem32) h->rem32 = dalloc<float>(H.ntree);
        for (int m = 0; m <= H.D; ++m) {
            const LevelArgs A = t->largs(m);
            launch_k(k_remainder, nblk(A.ncell / 8, OBLK), OBLK, 0, st, A, t->tables(), (const double*)h->c64[0],
                     h->C32(), h->rem32);
        }
        if (h->prm.bf16_coarse) {
            if (!h->d16) h->d16 = dalloc<float>(H.ncell);
            for (int m = H.mc; m <= H.D; ++m) {
                const LevelArgs A = t->largs(m);
                launch_k(k_diag_conservative<__nv_bfloat16>, nblk(A.ncell / 8, OBLK), OBLK, 0, st, A, t->tables(),
                         h->C64(), (const __nv_bfloat16*)h->c16[1], (const __nv_bfloat16*)h->c16[2],
                         (const __nv_bfloat16*)h->c16[3], (const float*)h->tw32, h->d16);
            }
        }
        ck_launch("convert");
        ck(cudaStreamSynchronize(st), "setup sync");
        for (int q = 0; q < 4; ++q) { dfree(h->c64[q]); h->c64[q] = nullptr; }
        dfree(h->tw64);
        h->tw64 = nullptr;
    }
    if (!h->beta) h->beta = dalloc<float>(H.nface);
    if (H.nface > 0)
        ck(cudaMemcpyAsync(h->beta, beta, H.nface * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy beta");
    ck(cudaStreamSynchronize(st), "setup sync");
}

int ocg_setup_hierarchy(const ocg_octree* t, const float* beta, const int32_t bc[6], const ocg_mg_params* prm,
                        void* stream, ocg_hier** out) {
    return guard([&] {
        if (!t || !beta || !bc || !prm || !out) throw Status(OCG_EINVAL, "null argument");
        *out = nullptr;
        if (prm->mu < 1 || prm->mu > 4 || prm->nu_pre < 0 || prm->nu_post < 0 || prm->nu_coarsest < 0 ||
            prm->mu_min_cells < 0 ||
            !(prm->alpha > 0) || !std::isfinite(prm->beta_restrict))
            throw Status(OCG_EINVAL, "invalid multigrid parameters");
        if (prm->coef_dtype != OCG_F64 && prm->coef_dtype != OCG_F32) throw Status(OCG_EINVAL, "coef_dtype");
        if (prm->coarsening != OCG_COARSEN_ALGEBRAIC && prm->coarsening != OCG_COARSEN_GEOMETRIC)
            throw Status(OCG_EINVAL, "coarsening");
        if (prm->coarsening == OCG_COARSEN_GEOMETRIC && t->H.desc.refine != OCG_REFINE_SDF_BAND)
            throw Status(OCG_EINVAL, "geometric coarsening needs an OCG_REFINE_SDF_BAND description");
        if (prm->reserved != 0) throw Status(OCG_EINVAL, "reserved must be 0");
        if (prm->sweep_form < OCG_SWEEP_AUTO || prm->sweep_form > OCG_SWEEP_TILE)
            throw Status(OCG_EINVAL, "sweep_form");
        if (t->H.D - t->H.mc + 1 > 2 * MAXLEV) throw Status(OCG_EINVAL, "too many levels");
        if (prm->bf16_coarse && prm->coef_dtype != OCG_F32) throw Status(OCG_EINVAL, "bf16_coarse needs F32");
        for (int q = 0; q < 6; ++q)
            if (bc[q] != OCG_BC_NEUMANN && bc[q] != OCG_BC_DIRICHLET) throw Status(OCG_EINVAL, "bc code");
        cudaStream_t st = (cudaStream_t)stream;
        const HostTree& H = t->H;
        t->upload();
        std::unique_ptr<ocg_hier> h(new ocg_hier());
        h->t = t;
        h->device = t->device;
        h->prm = *prm;
        bool ns = true;
        for (int q = 0; q < 6; ++q) {
            h->bc[q] = bc[q];
            if (bc[q] == OCG_BC_DIRICHLET) ns = false;
        }
        h->ns_auto = ns;
        build_coefficients(h.get(), beta, st);
        ensure_work(h.get());
        choose_tail(h.get(), 0, sizeof(float));
        choose_tail(h.get(), 1, sizeof(double));
        const int nlev = H.D - H.mc + 1;
        for (int q = 0; q < nlev; ++q) {
            h->sweep_form[q] = prm->sweep_form == OCG_SWEEP_AUTO ? OCG_SWEEP_OCTET : prm->sweep_form;
            h->tune_us[q][0] = h->tune_us[q][1] = h->tune_us[q][2] = h->tune_us[q][3] = -1.0;
        }
        if (prm->sweep_form == OCG_SWEEP_AUTO) {
            if (prm->coef_dtype == OCG_F64) autotune_sweeps<double>(h.get());
            else autotune_sweeps<float>(h.get());
        }
        // grid of the grid-stride reductions: 2 blocks per SM on small trees (few partials,
        // short latency chain), up to 8 per SM (full occupancy) once every thread has at
        // least 8 elements
        const int sms = sm_count();
        h->red_blocks = (int)std::max<int64_t>(2 * sms, std::min<int64_t>(8 * sms, H.ntree / (BLK * 8)));
        *out = h.release();
    });
}

void ocg_hier_destroy(ocg_hier* h) { delete h; }

int ocg_hier_update_beta(ocg_hier* h, const float* beta, void* stream) {
    return guard([&] {
        if (!h || !beta) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        cudaStream_t st = (cudaStream_t)stream;
        ck(cudaStreamSynchronize(st), "sync");
        build_coefficients(h, beta, st);
    });
}

int ocg_hier_export_coefs(const ocg_hier* h, int32_t m, double* c, double* cx, double* cy, double* cz) {
    return guard([&] {
        if (!h) throw Status(OCG_EINVAL, "null hierarchy");
        require_device(h);
        const HostTree& H = h->t->H;
        if (m < H.mc || m > H.D) throw Status(OCG_EINVAL, "level out of range");
        const LevelMeta& l = H.L(m);
        const std::vector<int64_t> cells = level_cells_morton(H, m);
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
            for (size_t e = 0; e < cells.size(); ++e) outs[q][e] = buf[cells[e] - l.off];
        }
    });
}

int ocg_hier_tuning(const ocg_hier* h, int32_t m, int32_t* form, double* us_octet, double* us_cell,
                    double* us_quad, double* us_tile) {
    return guard([&] {
        if (!h || !form || !us_octet || !us_cell || !us_quad || !us_tile) throw Status(OCG_EINVAL, "null argument");
        const HostTree& H = h->t->H;
        if (m < H.mc || m > H.D) throw Status(OCG_EINVAL, "level out of range");
        const int W = h->c64[0] ? 1 : 0;
        const bool in_tail = h->tail_top[W] != TAIL_NONE && m <= h->tail_top[W];
        *form = (in_tail || m == H.mc) ? -1 : h->sweep_form[m - H.mc];
        *us_octet = h->tune_us[m - H.mc][0];
        *us_cell = h->tune_us[m - H.mc][1];
        *us_quad = h->tune_us[m - H.mc][2];
        *us_tile = h->tune_us[m - H.mc][3];
    });
}

int ocg_apply_A(ocg_hier* h, int32_t dtype, const void* x, void* y, int32_t transpose, void* stream) {
    return guard([&] {
        if (!h || !x || !y) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        if (transpose != 0 && transpose != 1) throw Status(OCG_EINVAL, "transpose must be 0 or 1");
        if (transpose) ensure_adjoint(h);
        cudaStream_t st = (cudaStream_t)stream;
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        Ctx c{st, &h->probe, 0};
        auto run = [&](auto* tag, auto C) {
            using TO = std::remove_pointer_t<decltype(tag)>;
            using TC = typename CoefTypes<decltype(C)>::TC;
            using TW = typename CoefTypes<decltype(C)>::TW;
            TO* P = (TO*)h->xt;
            TO* Y = (TO*)h->yt;
            ck(cudaMemsetAsync(P, 0, H.ntree * sizeof(TO), st), "memset");
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_scatter<TO, TO>, nblk(H.nleaf), BLK, 0, st, (const TO*)x, P, t->leaf_cell, (int)H.nleaf);
            });
            if (transpose) apply_outer_T<TO, TC, TW>(h, C, P, Y, c);
            else apply_outer<TO, TC, TW>(h, C, P, Y, OP_NONE, c);
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_gather<TO, TO>, nblk(H.nleaf), BLK, 0, st, Y, (TO*)y, t->leaf_cell, (int)H.nleaf);
            });
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
        g_launches += c.count;
    });
}

int ocg_vcycle(ocg_hier* h, int32_t dtype, const void* r, void* z, void* stream) {
    return guard([&] {
        if (!h || !r || !z) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        cudaStream_t st = (cudaStream_t)stream;
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        Ctx c{st, &h->probe, 0};
        auto run = [&](auto* tag) {
            using TV = std::remove_pointer_t<decltype(tag)>;
            TV* U = (TV*)h->U;
            TV* B = (TV*)h->B;
            ck(cudaMemsetAsync(U, 0, cyc_len(H.ncell) * sizeof(TV), st), "memset");
            ck(cudaMemsetAsync(B, 0, cyc_len(H.ncell) * sizeof(TV), st), "memset");
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_scatter<TV, TV, true>, nblk(H.nleaf), BLK, 0, st, (const TV*)r, B, t->leaf_cell, (int)H.nleaf);
            });
            Cycle<TV>{h, U, B, c}.run();
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_gather<TV, TV, true>, nblk(H.nleaf), BLK, 0, st, U, (TV*)z, t->leaf_cell, (int)H.nleaf);
            });
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
        g_launches += c.count;
    });
}

int ocg_vcycle_transpose(ocg_hier* h, int32_t dtype, const void* z, void* r, void* stream) {
    return guard([&] {
        if (!h || !z || !r) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        cudaStream_t st = (cudaStream_t)stream;
        ensure_cycle_T(h);
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        Ctx c{st, &h->probe, 0};
        auto run = [&](auto* tag) {
            using TV = std::remove_pointer_t<decltype(tag)>;
            TV* U = (TV*)h->U;
            TV* B = (TV*)h->B;
            ck(cudaMemsetAsync(U, 0, H.ncell * sizeof(TV), st), "memset");
            ck(cudaMemsetAsync(B, 0, H.ncell * sizeof(TV), st), "memset");
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_scatter<TV, TV>, nblk(H.nleaf), BLK, 0, st, (const TV*)z, U, t->leaf_cell, (int)H.nleaf);
            });
            CycleT<TV>{h, U, B, (TV*)h->Xc, (TV*)h->UST, (TV*)h->Tacc, c}.run();
            launch(c, -1, 0, H.nleaf, [&] {
                launch_k(k_gather<TV, TV>, nblk(H.nleaf), BLK, 0, st, B, (TV*)r, t->leaf_cell, (int)H.nleaf);
            });
            ck_launch("vcycle_transpose");
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
        g_launches += c.count;
    });
}

int ocg_face_grad(ocg_hier* h, const double* p, const double* lambda, double* dbeta, void* stream) {
    return guard([&] {
        if (!h || !p || !lambda || !dbeta) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        const ocg_octree* t = h->t;
        const HostTree& H = t->H;
        if (H.nface == 0) return;
        ensure_adjoint(h);
        cudaStream_t st = (cudaStream_t)stream;
        Ctx c{st, nullptr, 0};
        // p into the tree cells with child means on inner cells (the pbar of Sec. 3.1),
        // lambda into the tree cells
        ck(cudaMemsetAsync(h->xt, 0, H.ntree * sizeof(double), st), "memset");
        ck(cudaMemsetAsync(h->yt, 0, H.ntree * sizeof(double), st), "memset");
        launch(c, -1, 0, H.nleaf, [&] {
            launch_k(k_scatter<double, double>, nblk(H.nleaf), BLK, 0, st, p, h->xt, t->leaf_cell, (int)H.nleaf);
        });
        launch(c, -1, 0, H.nleaf, [&] {
            launch_k(k_scatter<double, double>, nblk(H.nleaf), BLK, 0, st, lambda, h->yt, t->leaf_cell, (int)H.nleaf);
        });
        for (int m = H.D; m >= 1; --m) {
            const LevelArgs A = t->largs(m);
            launch(c, -1, m, A.ncell, [&] {
                if (h->c64[0])
                    launch_k(k_oavg<double, double>, nblk(A.ncell / 8, OBLK), OBLK, 0, st, A, t->tables(), h->c64[0], h->xt);
                else
                    launch_k(k_oavg<double, float>, nblk(A.ncell / 8, OBLK), OBLK, 0, st, A, t->tables(), h->c32[0], h->xt);
            });
        }
        launch(c, -1, 0, H.nface, [&] {
            FaceHs fh{};
            for (int d = 0; d <= H.D; ++d) fh.h[d] = 1.0 / (double)((int64_t)H.n0 << d);
            launch_k(k_face_grad, nblk(H.nface), BLK, 0, st, (int)H.nface, t->fminus, t->fplus, t->fkind, t->fdepth,
                                                      t->leaf_cell, t->level, t->oct_parent, fh, h->xt, h->yt, dbeta);
        });
        ck_launch("face_grad");
        g_launches += c.count;
    });
}

int ocg_pcg_solve(ocg_hier* h, const double* b, double* x, const ocg_solve_params* sp, ocg_solve_stats* stats,
                  void* stream) {
    int status = OCG_OK;
    int g = guard([&] {
        if (!h || !b || !x || !sp || !stats) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
        if (!(sp->tol > 0) || sp->max_iter < 1) throw Status(OCG_EINVAL, "tol must be > 0 and max_iter >= 1");
        if (sp->flags & ~(OCG_SOLVE_EAGER | OCG_SOLVE_TRANSPOSE | OCG_SOLVE_UNROLLED | OCG_SOLVE_BICGSTAB | OCG_SOLVE_WARM))
            throw Status(OCG_EINVAL, "unknown solve flags");
        cudaStream_t st = (cudaStream_t)stream;
        const bool tr = (sp->flags & OCG_SOLVE_TRANSPOSE) != 0;
        const bool bi = tr && (sp->flags & OCG_SOLVE_BICGSTAB) != 0;
        if (bi) ensure_bicg(h);
        else if (tr) { ensure_adjoint(h); ensure_cycle_T(h); }
        switch (sp->precision) {
            case OCG_PREC_FP64:
                if (!h->c64[0]) throw Status(OCG_EINVAL, "FP64 solve needs coef_dtype F64");
                status = bi   ? krylov_solve<BiCG, double, double>(h, h->C64(), 0, b, x, sp, stats, st)
                            : tr ? krylov_solve<PcgT, double, double>(h, h->C64(), 0, b, x, sp, stats, st)
                                 : krylov_solve<Pcg, double, double>(h, h->C64(), 0, b, x, sp, stats, st);
                break;
            case OCG_PREC_FP32:
                if (!h->c32[0]) throw Status(OCG_EINVAL, "FP32 solve needs coef_dtype F32");
                status = bi   ? krylov_solve<BiCG, float, float>(h, h->C32(), 1, b, x, sp, stats, st)
                            : tr ? krylov_solve<PcgT, float, float>(h, h->C32(), 1, b, x, sp, stats, st)
                                 : krylov_solve<Pcg, float, float>(h, h->C32(), 1, b, x, sp, stats, st);
                break;
            case OCG_PREC_MIXED:
                if (!h->c32[0]) throw Status(OCG_EINVAL, "mixed solve needs coef_dtype F32");
                status = bi   ? krylov_solve<BiCG, double, float>(h, h->C32(), 2, b, x, sp, stats, st)
                            : tr ? krylov_solve<PcgT, double, float>(h, h->C32(), 2, b, x, sp, stats, st)
                                 : krylov_solve<Pcg, double, float>(h, h->C32(), 2, b, x, sp, stats, st);
                break;
            default:
                throw Status(OCG_EINVAL, "precision");
        }
    });
    return g != OCG_OK ? g : status;
}

int ocg_probe_set(ocg_hier* h, int32_t kind, int32_t level) {
    return guard([&] {
        if (!h) throw Status(OCG_EINVAL, "null hierarchy");
        require_device(h);
        if (kind < OCG_PROBE_OFF || kind > OCG_PROBE_TAIL) throw Status(OCG_EINVAL, "probe kind");
        h->probe.kind = kind;
        h->probe.level = level;
        h->probe.used = 0;
    });
}

int ocg_probe_read(ocg_hier* h, void* stream, int64_t* launches, double* total_ms, int64_t* cells) {
    return guard([&] {
        if (!h || !launches || !total_ms || !cells) throw Status(OCG_EINVAL, "null argument");
        require_device(h);
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

int ocg_set_allocator(ocg_alloc_fn alloc, ocg_free_fn free_fn, void* ctx) {
    return guard([&] {
        if ((alloc == nullptr) != (free_fn == nullptr)) throw Status(OCG_EINVAL, "give both hooks or neither");
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        g_hooks.alloc = alloc;
        g_hooks.free = free_fn;
        g_hooks.ctx = alloc ? ctx : nullptr;
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
#include "batch_host.cuh"

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
        require_device(h);
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
        Ctx c{st, nullptr, 0};
        launch(c, -1, 0, H.nleaf, [&] {
            launch_k(k_scatter<float, float>, nblk(H.nleaf), BLK, 0, st, x, P, t->leaf_cell, (int)H.nleaf);
        });
        ck_launch("scatter");
        if (h->c64[0]) apply_outer<float, double, double>(h, h->C64(), P, Y, OP_NONE, c);
        else apply_outer<float, float, float>(h, h->C32(), P, Y, OP_NONE, c);
        launch(c, -1, 0, H.nleaf, [&] {
            launch_k(k_gather<float, float>, nblk(H.nleaf), BLK, 0, st, Y, y, t->leaf_cell, (int)H.nleaf);
        });
        ck_launch("gather");
        g_launches += c.count;
    });
}
