// Host side of the batched form (included by ocg_api.cu after the hierarchy types).
//
// The level at height g of a problem is visited together with the levels at height g of
// the others.  W-cycles align the problems at their finest levels (height H), so that the
// recursion of Alg. 4 (mu visits of the next height per visit) is one schedule for all,
// and a problem whose coarse tail sits at height g runs it there (one CTA per problem, one
// launch per height that holds tails); V-cycles align them at their tails (height 0), and
// all tails run in one launch.  A launch lists
// its (problem, level) work items; a block map sends every block to its item.  The sweep
// form of each height (thread per octet or per cell) is timed at set-up, the faster kept.
// The whole PCG loop is one CUDA graph with a WHILE node whose condition is "some problem
// has not converged"; converged problems are frozen (their blocks return at once).

struct ocg_batch {
    struct Map {
        int w0 = 0, nw = 0;     // work items in dW
        int i0 = 0, nb = 0;     // block map in dI, blocks of the launch
    };
    struct Phase {
        Map oct, cell;          // the same items mapped for the two sweep forms
    };
    int n = 0;
    std::vector<ocg_hier*> hs;
    ocg_mg_params prm{};
    int H = 0, Dmax = 0;
    BProb* dP = nullptr;
    BWork* dW = nullptr;
    int* dI = nullptr;
    std::vector<Phase> down, up, fixb;   // index g = 1..H (height)
    std::vector<Map> tails;              // index g = 0..H: the coarse tails at height g
    std::vector<Map> avg;                // index m = 1..Dmax
    Map apply;
    int mu = 1;
    Map vec;                             // vector kernels (items unused)
    int tail_nt = 32;
    size_t tail_smem = 0;
    std::vector<int> form;               // per height
    std::vector<std::array<double, 2>> tune_us;
    double* S = nullptr;                 // n x S_COUNT
    double* hS = nullptr;                // pinned mirror
    double* part = nullptr;
    unsigned* cnt = nullptr;
    unsigned* gcnt = nullptr;
    BIO* dio = nullptr;
    BIO* hio = nullptr;                  // pinned
    cudaStream_t cap = nullptr;
    GraphSolve gs;

    ~ocg_batch() {
        if (gs.exec) cudaGraphExecDestroy(gs.exec);
        if (gs.graph) cudaGraphDestroy(gs.graph);
        if (cap) cudaStreamDestroy(cap);
        dfree(dP); dfree(dW); dfree(dI); dfree(S); dfree(part); dfree(cnt); dfree(gcnt); dfree(dio);
        if (hS) cudaFreeHost(hS);
        if (hio) cudaFreeHost(hio);
    }
};

namespace {

struct BatchBuild {
    std::vector<BWork> W;
    std::vector<int> I;
    // items: (problem, level, flags); cells per block of the form
    ocg_batch::Map map(const std::vector<std::array<int, 3>>& items, const std::vector<BProb>& P, int cells_per_block) {
        ocg_batch::Map M;
        M.w0 = (int)W.size();
        M.nw = (int)items.size();
        M.i0 = (int)I.size();
        int b = 0;
        for (size_t k = 0; k < items.size(); ++k) {
            const BProb& pr = P[items[k][0]];
            const int ncell = pr.L[items[k][1] - pr.mc].ncell;
            const int nb = (ncell + cells_per_block - 1) / cells_per_block;
            W.push_back(BWork{items[k][0], items[k][1], b, items[k][2]});
            for (int q = 0; q < nb; ++q) I.push_back(M.w0 + (int)k);
            b += nb;
        }
        M.nb = b;
        return M;
    }
};

struct BatchRun {
    ocg_batch* bt;
    Ctx& c;
    cudaGraphConditionalHandle cond;
    int set_cond;

    BRed red(int op, bool sc = false) const { return BRed{op, bt->n, bt->gcnt, cond, sc ? set_cond : 0}; }
    const int* I(const ocg_batch::Map& M) const { return bt->dI + M.i0; }
    template <class F>
    void go(int64_t cells, F&& f) {
        launch(c, -1, 0, cells, f);
        ck_launch("batched launch");
    }
    void sweep(int h, int colour, bool last_post, int form, int skip_first = 0) {
        const ocg_batch::Phase& ph = last_post ? bt->up[h] : bt->down[h];
        if (form == OCG_SWEEP_CELL)
            go(0, [&] { kb_csweep<<<ph.cell.nb, BLK, 0, c.st>>>(bt->dP, bt->dW, I(ph.cell), colour, skip_first); });
        else
            go(0, [&] { kb_osweep<<<ph.oct.nb, OBLK, 0, c.st>>>(bt->dP, bt->dW, I(ph.oct), colour, 0, skip_first); });
    }
    // Alg. 4 at height g for every problem with a level there; fas: first visit after a
    // restriction from above, prolong_up: the last visit, whose final operation prolongs
    // onto height g + 1
    void cyc(int g, bool fas, bool prolong_up) {
        const ocg_mg_params& P = bt->prm;
        const float scale = (float)(P.beta_restrict / P.alpha);
        const ocg_batch::Map& tl = bt->tails[g];
        if (tl.nw > 0)
            go(0, [&] {
                kb_otail<<<tl.nw, bt->tail_nt, bt->tail_smem, c.st>>>(bt->dP, bt->dW + tl.w0, scale, fas ? 1 : 0,
                                                                         prolong_up ? 1 : 0);
            });
        if (g < 1 || bt->down[g].oct.nw == 0) return;
        const ocg_batch::Phase& f = bt->fixb[g];
        if (fas && f.oct.nw > 0)
            go(0, [&] { kb_osweep<<<f.oct.nb, OBLK, 0, c.st>>>(bt->dP, bt->dW, I(f.oct), 0, 1, 0); });
        for (int it = 0; it < P.nu_pre; ++it) {
            // a problem's finest level is visited once per cycle, and its first sweep there
            // was formed by the vector kernels (fuse_first)
            sweep(g, 0, false, bt->form[g], it == 0 ? 1 : 0);
            sweep(g, 1, false, bt->form[g]);
        }
        const ocg_batch::Map& d = bt->down[g].oct;
        go(0, [&] { kb_orestrict<<<d.nb, OBLK, 0, c.st>>>(bt->dP, bt->dW, I(d), scale); });
        for (int k = 0; k < bt->mu; ++k) cyc(g - 1, k == 0, k == bt->mu - 1);
        for (int it = 0; it < P.nu_post; ++it) {
            sweep(g, 1, false, bt->form[g]);
            sweep(g, 0, prolong_up && it == P.nu_post - 1, bt->form[g]);
        }
    }
    void cycle() {
        go(0, [&] { kb_zero_u<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec)); });
        cyc(bt->H, false, false);
    }
    void apply(int which) {
        for (int m = bt->Dmax; m >= 1; --m) {
            const ocg_batch::Map& a = bt->avg[m];
            if (a.nw > 0) go(0, [&] { kb_oavg<<<a.nb, OBLK, 0, c.st>>>(bt->dP, bt->dW, I(a), which); });
        }
        go(0, [&] {
            kb_oapply<<<bt->apply.nb, OBLK2, 0, c.st>>>(bt->dP, bt->dW, I(bt->apply), which, red(OP_ALPHA));
        });
    }
    void half_a() {
        apply(0);
        go(0, [&] { kb_update<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), red(OP_RR, true)); });
        go(0, [&] { kb_project<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec)); });
    }
    void begin() {
        go(0, [&] { kb_begin<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), bt->dio, red(OP_BB)); });
        go(0, [&] { kb_rinit<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec)); });
        cycle();
        go(0, [&] { kb_dot_rz<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), red(OP_RZ0)); });
        go(0, [&] { kb_pupdate<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), 1); });
        half_a();
    }
    void body() {
        cycle();
        go(0, [&] { kb_dot_rz<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), red(OP_BETA)); });
        go(0, [&] { kb_pupdate<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), 0); });
        half_a();
    }
    void finish() {
        go(0, [&] { kb_copy_x<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec)); });
        apply(1);
        go(0, [&] { kb_resid<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), red(OP_TRUE)); });
        go(0, [&] { kb_xsum<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), red(OP_XMEAN)); });
        go(0, [&] { kb_gather<<<bt->vec.nb, BLK, 0, c.st>>>(bt->dP, I(bt->vec), bt->dio); });
    }
};

// time 20 colour sweeps of height h in each form (graph replays), keep the faster
void batch_autotune(ocg_batch* bt) {
    if (!bt->cap) ck(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t cs = bt->cap;
    for (ocg_hier* h : bt->hs) {
        ck(cudaMemsetAsync(h->U, 0, cyc_len(h->t->H.ncell) * sizeof(float), cs), "memset");
        ck(cudaMemsetAsync(h->B, 0, cyc_len(h->t->H.ncell) * sizeof(float), cs), "memset");
    }
    ck(cudaMemsetAsync(bt->S, 0, (size_t)bt->n * S_COUNT * sizeof(double), cs), "memset");
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "cudaEventCreate");
    ck(cudaEventCreate(&e1), "cudaEventCreate");
    for (int h = 1; h <= bt->H; ++h) {
        for (int form = 0; form < 2; ++form) {
            Ctx c{cs, nullptr, 0};
            BatchRun br{bt, c, 0, 0};
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int q = 0; q < 20; ++q) br.sweep(h, q & 1, false, form);
            ck(cudaStreamEndCapture(cs, &g), "end capture");
            ck(cudaGraphInstantiate(&ge, g, 0), "graph instantiate");
            for (int w = 0; w < 2; ++w) ck(cudaGraphLaunch(ge, cs), "graph launch");
            ck(cudaEventRecord(e0, cs), "event");
            for (int r = 0; r < 5; ++r) ck(cudaGraphLaunch(ge, cs), "graph launch");
            ck(cudaEventRecord(e1, cs), "event");
            ck(cudaEventSynchronize(e1), "event sync");
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            bt->tune_us[h][form] = ms * 1000.0 / (5 * 20);
            cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
        }
        bt->form[h] = bt->tune_us[h][1] < bt->tune_us[h][0] ? OCG_SWEEP_CELL : OCG_SWEEP_OCTET;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

void batch_build_graph(ocg_batch* bt) {
    if (!bt->cap) ck(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t cs = bt->cap;
    GraphSolve& gs = bt->gs;
    Ctx c{cs, nullptr, 0};
    ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus stt;
    try {
        ck(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
        cudaGraphConditionalHandle cond;
        ck(cudaGraphConditionalHandleCreate(&cond, g, 0, 0), "conditional handle");
        BatchRun br{bt, c, cond, 1};
        br.begin();
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
        br.finish();
        gs.outer_kernels = c.count;
        ck(cudaStreamEndCapture(cs, &g), "end capture");
        Ctx cb{cs, nullptr, 0};
        ck(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
           "begin body capture");
        BatchRun bb{bt, cb, cond, 1};
        bb.body();
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

}  // namespace

extern "C" {

int ocg_batch_create(ocg_hier* const* hs, int32_t n, void* stream, ocg_batch** out) {
    return guard([&] {
        if (!hs || !out || n < 1) throw Status(OCG_EINVAL, "null argument or n < 1");
        *out = nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        std::unique_ptr<ocg_batch> bt(new ocg_batch());
        bt->n = n;
        if (!hs[0]) throw Status(OCG_EINVAL, "null hierarchy");
        bt->prm = hs[0]->prm;
        bt->mu = bt->prm.mu;
        std::vector<BProb> P(n);
        int vb = 0, ab = 0;
        std::vector<int> tops(n);
        for (int p = 0; p < n; ++p) {
            ocg_hier* h = hs[p];
            if (!h) throw Status(OCG_EINVAL, "null hierarchy");
            require_device(h);
            for (int q = 0; q < p; ++q)
                if (hs[q] == h) throw Status(OCG_EINVAL, "a hierarchy appears twice in the batch");
            const ocg_mg_params& m = h->prm;
            if (!h->c32[0] || m.bf16_coarse) throw Status(OCG_EINVAL, "batched solves need FP32 coefficients");
            if (m.mu < 1 || m.mu > 2 || m.mu != bt->prm.mu || m.mu_min_cells != 0 || m.nu_post < 1 ||
                m.nu_pre != bt->prm.nu_pre || m.nu_post != bt->prm.nu_post ||
                m.nu_coarsest != bt->prm.nu_coarsest || m.alpha != bt->prm.alpha ||
                m.beta_restrict != bt->prm.beta_restrict)
                throw Status(OCG_EINVAL, "batched solves need V- or W-cycles (mu 1 or 2, mu_min_cells 0, "
                                         "nu_post >= 1) with equal parameters");
            if (h->tail_top[0] == TAIL_NONE) throw Status(OCG_EINVAL, "every problem needs a shared-memory coarse tail");
            bt->hs.push_back(h);
            const ocg_octree* t = h->t;
            const HostTree& Ht = t->H;
            BProb& b = P[p];
            std::memset(&b, 0, sizeof(b));
            b.T = t->tables();
            b.C = h->C32();
            b.U = (float*)h->U;
            b.B = (float*)h->B;
            b.x = h->x; b.r = h->r; b.p = h->p; b.Ap = h->Ap; b.bt = h->bt; b.xt = h->xt; b.yt = h->yt;
            b.flags = t->flags;
            b.rem = h->rem32;
            b.leaf_cell = t->leaf_cell;
            b.ntree = (int)Ht.ntree;
            b.nleaf = (int)Ht.nleaf;
            b.D = Ht.D;
            b.mc = Ht.mc;
            b.fuse_first = first_sweep_fusable(h) ? 1 : 0;
            for (int m2 = Ht.mc; m2 <= Ht.D; ++m2)
                b.L[m2 - Ht.mc] = BLev{(int)Ht.L(m2).off, (int)Ht.L(m2).ncell, Ht.L(m2).ni};
            b.tail = h->tail_args[0];
            b.nbv = (int)std::max<int64_t>(1, std::min<int64_t>(256, (Ht.ntree + 16 * BLK - 1) / (16 * BLK)));
            b.vb0 = vb;
            vb += b.nbv;
            int na = 0;
            for (int m2 = 0; m2 <= Ht.D; ++m2) na += (int)nblk(Ht.L(m2).ncell / 8, OBLK);
            b.nba = na;
            b.ab0 = ab;
            ab += na;
            tops[p] = h->tail_top[0];
            bt->H = std::max(bt->H, Ht.D - tops[p]);
            bt->Dmax = std::max(bt->Dmax, Ht.D);
            bt->tail_smem = std::max(bt->tail_smem, h->tail_smem[0]);
            const int noct = h->tail_args[0].L[0].ni * h->tail_args[0].L[0].ni * h->tail_args[0].L[0].ni;
            bt->tail_nt = std::max(bt->tail_nt, std::min(512, (noct + 31) / 32 * 32));
        }
        // scalars, partials, counters
        int maxnb = 1;
        for (const BProb& b : P) maxnb = std::max(maxnb, std::max(b.nbv, b.nba));
        bt->S = dalloc<double>((int64_t)n * S_COUNT);
        ck(cudaMallocHost((void**)&bt->hS, (size_t)n * S_COUNT * sizeof(double)), "cudaMallocHost");
        bt->part = dalloc<double>((int64_t)n * 3 * maxnb);
        bt->cnt = dalloc<unsigned>(n);
        bt->gcnt = dalloc<unsigned>(1);
        ck(cudaMemsetAsync(bt->cnt, 0, n * sizeof(unsigned), st), "memset");
        ck(cudaMemsetAsync(bt->gcnt, 0, sizeof(unsigned), st), "memset");
        bt->dio = dalloc<BIO>(n);
        ck(cudaMallocHost((void**)&bt->hio, n * sizeof(BIO)), "cudaMallocHost");
        for (int p = 0; p < n; ++p) {
            P[p].S = bt->S + (int64_t)p * S_COUNT;
            P[p].part = bt->part + (int64_t)p * 3 * maxnb;
            P[p].cnt = bt->cnt + p;
            // inner cells of bt stay 0 (single solves zero bt before scattering too)
            ck(cudaMemsetAsync(P[p].bt, 0, P[p].ntree * sizeof(double), st), "memset");
        }
        // work lists
        BatchBuild bb;
        // heights: for mu = 2 every problem's finest level sits at H (level m of problem p
        // at height g = H - (D_p - m)), so that the recursion visits each problem's levels
        // as its own cycle does; for mu = 1 the tails sit at height 0 (m = tops[p] + g), so
        // that all tails run in one launch.  A tail item's flag marks a tail that is the
        // problem's finest level (no restriction into it, no prolongation out of it).
        bt->down.resize(bt->H + 1);
        bt->up.resize(bt->H + 1);
        bt->fixb.resize(bt->H + 1);
        bt->tails.resize(bt->H + 1);
        for (int g = 0; g <= bt->H; ++g) {
            std::vector<std::array<int, 3>> dn, upl, fx, tl;
            for (int p = 0; p < n; ++p) {
                const int m = bt->mu == 1 ? tops[p] + g : P[p].D - (bt->H - g);
                if (m < tops[p] || m > P[p].D) continue;
                if (m == tops[p]) {
                    tl.push_back({p, m, m == P[p].D ? 1 : 0});
                    continue;
                }
                dn.push_back({p, m, 0});
                upl.push_back({p, m, m < P[p].D ? 1 : 0});
                if (m < P[p].D) fx.push_back({p, m, 2});
            }
            bt->tails[g] = bb.map(tl, P, 1 << 30);   // one block per problem
            if (g == 0) continue;
            bt->down[g].oct = bb.map(dn, P, 8 * OBLK);
            bt->down[g].cell = bb.map(dn, P, BLK);
            bt->up[g].oct = bb.map(upl, P, 8 * OBLK);
            bt->up[g].cell = bb.map(upl, P, BLK);
            bt->fixb[g].oct = bb.map(fx, P, 8 * OBLK);
        }
        bt->avg.resize(bt->Dmax + 1);
        for (int m = 1; m <= bt->Dmax; ++m) {
            std::vector<std::array<int, 3>> it;
            for (int p = 0; p < n; ++p)
                if (P[p].D >= m) it.push_back({p, m, 0});
            bt->avg[m] = bb.map(it, P, 8 * OBLK);
        }
        {
            std::vector<std::array<int, 3>> it;
            for (int p = 0; p < n; ++p)
                for (int m = 0; m <= P[p].D; ++m) it.push_back({p, m, 0});
            bt->apply = bb.map(it, P, 8 * OBLK);
        }
        bt->vec.i0 = (int)bb.I.size();
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < P[p].nbv; ++q) bb.I.push_back(p);
        bt->vec.nb = vb;
        bt->dW = dupload(bb.W);
        bt->dI = dupload(bb.I);
        bt->dP = dupload(P);
        ck(cudaFuncSetAttribute(kb_otail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->tail_smem),
           "cudaFuncSetAttribute");
        ck(cudaStreamSynchronize(st), "batch setup sync");
        bt->form.assign(bt->H + 1, OCG_SWEEP_OCTET);
        bt->tune_us.assign(bt->H + 1, {-1.0, -1.0});
        if (bt->prm.sweep_form == OCG_SWEEP_AUTO) batch_autotune(bt.get());
        else for (int h = 1; h <= bt->H; ++h) bt->form[h] = bt->prm.sweep_form;
        ck(cudaStreamSynchronize(bt->cap ? bt->cap : st), "batch setup sync");
        *out = bt.release();
    });
}

void ocg_batch_destroy(ocg_batch* b) { delete b; }

int ocg_batch_info(const ocg_batch* b, int32_t h, int32_t* heights, int32_t* form, double* us_octet,
                   double* us_cell) {
    return guard([&] {
        if (!b || !heights || !form || !us_octet || !us_cell) throw Status(OCG_EINVAL, "null argument");
        *heights = b->H;
        if (h < 1 || h > b->H) throw Status(OCG_EINVAL, "height out of range");
        *form = b->form[h];
        *us_octet = b->tune_us[h][0];
        *us_cell = b->tune_us[h][1];
    });
}

int ocg_pcg_solve_batched(ocg_batch* bt, const double* const* b, double* const* x, const ocg_solve_params* sp,
                          ocg_solve_stats* stats, void* stream) {
    int status = OCG_OK;
    const int g = guard([&] {
        if (!bt || !b || !x || !sp || !stats) throw Status(OCG_EINVAL, "null argument");
        if (!(sp->tol > 0) || sp->max_iter < 1) throw Status(OCG_EINVAL, "tol must be > 0 and max_iter >= 1");
        if (sp->precision != OCG_PREC_MIXED) throw Status(OCG_EINVAL, "batched solves run in mixed precision");
        if (sp->flags != 0) throw Status(OCG_EINVAL, "batched solves take no flags");
        require_device(bt->hs[0]);
        cudaStream_t st = (cudaStream_t)stream;
        const int n = bt->n;
        for (int p = 0; p < n; ++p) {
            if (!b[p] || !x[p]) throw Status(OCG_EINVAL, "null vector");
            double* S = bt->hS + (int64_t)p * S_COUNT;
            std::memset(S, 0, S_COUNT * sizeof(double));
            const bool ns = sp->nullspace < 0 ? bt->hs[p]->ns_auto : sp->nullspace != 0;
            S[S_NS] = ns ? 1.0 : 0.0;
            S[S_TOL] = sp->tol;
            S[S_MAXIT] = sp->max_iter;
            bt->hio[p] = BIO{b[p], x[p]};
        }
        ck(cudaMemcpyAsync(bt->S, bt->hS, (size_t)n * S_COUNT * sizeof(double), cudaMemcpyHostToDevice, st),
           "copy scalars");
        ck(cudaMemcpyAsync(bt->dio, bt->hio, n * sizeof(BIO), cudaMemcpyHostToDevice, st), "copy vectors");
        if (!bt->gs.exec) batch_build_graph(bt);
        ck(cudaGraphLaunch(bt->gs.exec, st), "graph launch");
        ck(cudaMemcpyAsync(bt->hS, bt->S, (size_t)n * S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st),
           "copy scalars");
        ck(cudaStreamSynchronize(st), "stream sync");
        int kmax = 0;
        bool all = true, finite = true;
        for (int p = 0; p < n; ++p) {
            const double* S = bt->hS + (int64_t)p * S_COUNT;
            ocg_solve_stats& o = stats[p];
            std::memset(&o, 0, sizeof(o));
            const int k = (int)S[S_K];
            kmax = std::max(kmax, k);
            const double bb = S[S_BB];
            o.iterations = k;
            o.hist[0] = 1.0;
            for (int q = 1; q <= k && q < OCG_HIST; ++q) o.hist[q] = S[S_HIST + q];
            o.rel_res = bb > 0.0 ? std::sqrt(std::max(S[S_RR], 0.0) / bb) : 0.0;
            o.true_rel_res = bb > 0.0 ? std::sqrt(std::max(S[S_TRUE], 0.0) / bb) : 0.0;
            o.converged = !(o.rel_res > sp->tol) ? 1 : 0;
            all = all && o.converged;
            finite = finite && std::isfinite(o.rel_res) && std::isfinite(o.true_rel_res);
        }
        const int64_t kernels = bt->gs.outer_kernels + (int64_t)std::max(kmax - 1, 0) * bt->gs.body_kernels;
        for (int p = 0; p < n; ++p) stats[p].kernels = kernels;
        g_launches += kernels;
        if (!finite) {
            status = OCG_ENAN;
            g_err = "non-finite residual norm";
        } else if (!all) {
            status = OCG_ENOTCONV;
            g_err = "a problem of the batch reached max_iter before the tolerance";
        }
    });
    return g != OCG_OK ? g : status;
}

}  // extern "C"
