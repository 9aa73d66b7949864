// qai_batched.cu -- many fields in one call (see include/qai.h).
//
// Rank-2 and rank-3 fields run as persistent grouped launches: each kernel of
// the plain launch sequence (step A, the local first EDT with its separable
// fallback, the signed-point route with the dense second EDT behind it) runs
// once for all of them, its resident CTAs taking (field, virtual block) work
// items from a device cursor in queue order (GroupQueue). Fields share a
// launch when they share the kernel's tile shape; a field whose gate flag is
// clear when the launch starts adds no work items, so the fallbacks cost a
// batch a few launches, not a few per field. Rank-1 fields run as two grouped
// row passes. The launch sequence -- the argument tables copied in, the
// cursors and route counters cleared, then the grouped kernels -- is captured
// into a CUDA graph once and replayed. An autotuner times the batch itself to
// pick the queue order (largest field first or as given), the points per
// work item of the grid-stride kernels and the column tiles (width, band
// height), and caches them by the batch's shapes. With a route-selection
// flag, or inside a caller's stream capture, rank-2 and rank-3 fields run
// their own plain sequences on forked streams instead.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "qai.h"
#include "qai_host.h"
#include "qai_launch.h"

using namespace qai;
using namespace qai::host;

namespace {

struct GroupCfg {
    int order = 1;    // 0: as given, 1: largest field first
    int streams = 4;  // rank 2 and 3: streams the fields' launch sequences are dealt onto
};
constexpr int kMaxStreams = 8;

// Streams forked from a caller's stream (an event recorded there, waited on
// by each) and joined back (one event per stream, waited on by the caller's
// stream). Works inside a stream capture: the forked streams join it.
struct Forker {
    cudaStream_t s[kMaxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxStreams] = {};
    bool ok = false;
};
Forker* forker()
{
    thread_local Forker f;
    if (!f.ok) {
        bool good = cudaEventCreateWithFlags(&f.fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; good && i < kMaxStreams; ++i)
            good = cudaStreamCreateWithFlags(&f.s[i], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&f.join_ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!good) return nullptr;
        f.ok = true;
    }
    return &f;
}

struct Field {
    int index;
    Shape sh;
    Layout lay;
    size_t ws_off;
    const int32_t* q;
    float* out;
    MethodArgs m;
};

struct Batch {
    std::vector<Field> f;
    std::vector<int> group[4];  // field positions per rank
    size_t header = 0;          // grouped launches' cursors, counters and argument tables
    size_t ws_total = 0;
    bool grouped = false;       // rank 2 and 3 as grouped launches
};

// The argument tables of one field's grouped launches at most (every kernel
// of the plain sequence once), the cursors, and the route counters.
constexpr int kLaunchesPerField = 32;
size_t header_bytes(int n)
{
    const size_t tables = (size_t)n * (6 * sizeof(LocalArgs) + 7 * sizeof(RouteArgs) + 2 * sizeof(RowArgs) +
                                       4 * sizeof(ColArgs));
    return align256((size_t)(kLaunchesPerField * n + 64) * 4) + align256((size_t)n * kCtrWords * 4) +
           align256(tables);
}

std::mutex g_mu;
std::unordered_map<uint64_t, GroupCfg> g_tuned;  // group signature -> config
struct GraphEntry {
    uint64_t key;
    cudaGraphExec_t exec;
    int kernels;
    void* host_tables;  // pinned image of the grouped launches' argument tables (copied in by the graph)
};
std::vector<GraphEntry> g_graphs;  // most recent last
constexpr size_t kMaxGraphs = 16;

uint64_t fnv(const void* p, size_t n, uint64_t h)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

uint64_t group_signature(const Batch& bt, int rank)
{
    std::vector<int64_t> v;
    for (int i : bt.group[rank]) {
        v.push_back(bt.f[i].sh.nz);
        v.push_back(bt.f[i].sh.ny);
        v.push_back(bt.f[i].sh.nx);
    }
    std::sort(v.begin(), v.end());
    uint64_t h = fnv(&rank, sizeof rank, 1469598103934665603ull);
    return fnv(v.data(), v.size() * sizeof(int64_t), h);
}

GroupCfg tuned_cfg(uint64_t sig)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(sig);
    return it == g_tuned.end() ? GroupCfg() : it->second;
}

qai_status plan(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                const int64_t* dims, const double* eb, const qai_params* params, Batch& bt)
{
    if (n < 1) return fail(QAI_ERR_INVALID_ARG, "n must be >= 1");
    if (!d_q || !d_out || !ranks || !dims || !eb) return fail(QAI_ERR_INVALID_ARG, "NULL array argument");
    qai_params defaults;
    qai_default_params(&defaults);
    const qai_params* p = params ? params : &defaults;
    qai_status s = check_params(p);
    if (s != QAI_OK) return s;
    bt.f.resize(n);
    bt.header = header_bytes(n);
    bt.grouped = (p->flags & (QAI_FLAG_EDT2_DENSE | QAI_FLAG_EDT2_HANDOVER | QAI_FLAG_EDT2_LIST |
                              QAI_FLAG_EDT1_SEPARABLE)) == 0;
    size_t off = bt.header;
    for (int i = 0; i < n; ++i) {
        Field& f = bt.f[i];
        f.index = i;
        if ((s = make_shape(ranks[i], dims + 3 * i, &f.sh)) != QAI_OK) return s;
        if (!d_q[i] || !d_out[i]) return fail(QAI_ERR_INVALID_ARG, "field %d: NULL buffer", i);
        if (!(eb[i] > 0.0) || !std::isfinite(eb[i])) return fail(QAI_ERR_INVALID_ARG, "field %d: bad eb", i);
        f.lay = layout_for(f.sh, 0);
        f.ws_off = off;
        off = align256(off + f.lay.total);
        f.q = d_q[i];
        f.out = d_out[i];
        f.m = method_args(p, eb[i]);
        bt.group[f.sh.rank].push_back(i);
    }
    bt.ws_total = off;
    return QAI_OK;
}

// Rank-1 fields: the grouped row passes (phase 1 writes Dist1 and S, phase 2
// GetBoundary(S), the EDT of B2 and step E), at most kMaxGroup fields a launch.
qai_status launch_rank1(const Batch& bt, const std::vector<int>& order, char* ws, cudaStream_t st, int* kernels)
{
    for (size_t c0 = 0; c0 < order.size(); c0 += kMaxGroup) {
        const int cn = (int)std::min(order.size() - c0, (size_t)kMaxGroup);
        auto F = [&](int k) -> const Field& { return bt.f[order[c0 + k]]; };
        int max_nx = 0;
        for (int k = 0; k < cn; ++k) max_nx = std::max(max_nx, F(k).sh.nx);
        for (int phase = 1; phase <= 2; ++phase) {
            thread_local RowTable rt;  // large: built on the host, copied into the launch
            std::memset(&rt, 0, sizeof rt);
            rt.n = cn;
            rt.smem_nx = max_nx;
            rt.warps = rowpass_warps(max_nx);
            int acc = 0;
            for (int k = 0; k < cn; ++k) {
                const Field& f = F(k);
                char* b = ws + f.ws_off;
                RowArgs r{};
                r.rank = 1; r.nz = f.sh.nz; r.ny = f.sh.ny; r.nx = f.sh.nx;
                r.q = f.q; r.eqm = reinterpret_cast<uint8_t*>(b + f.lay.eqm); r.m = f.m;
                int32_t* dist1 = reinterpret_cast<int32_t*>(b + f.lay.dist1);
                int8_t* s = reinterpret_cast<int8_t*>(b + f.lay.s);
                if (phase == 1) {
                    r.dist1 = dist1; r.s_out = s;
                } else {
                    r.s_in = s; r.dist1_in = dist1; r.out = f.out;
                }
                prepare_rowpass(r);
                rt.args[k] = r;
                rt.first_row[k] = acc;
                acc += f.sh.nz * f.sh.ny;
            }
            rt.first_row[cn] = acc;
            cudaError_t e = launch_rowpass_grouped(phase, true, rt, st);
            ++*kernels;
            if (e != cudaSuccess) return cuda_fail(e, "grouped row pass");
        }
    }
    return QAI_OK;
}

// The launches of one rank group on `st` (rank 2 and 3: on cfg.streams
// streams forked from it and joined back). Adds the kernels launched to
// *kernels.
qai_status launch_group(const Batch& bt, int rank, const GroupCfg& cfg, char* ws, cudaStream_t st,
                        int* kernels)
{
    std::vector<int> order = bt.group[rank];
    if (order.empty()) return QAI_OK;
    if (cfg.order == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return bt.f[a].sh.N > bt.f[b].sh.N; });
    if (rank == 1) return launch_rank1(bt, order, ws, st, kernels);
    const int ns = std::max(1, std::min(cfg.streams, kMaxStreams));
    Forker* fk = ns > 1 ? forker() : nullptr;
    if (ns > 1 && !fk) return cuda_fail(cudaGetLastError(), "batch streams");
    cudaError_t e;
    if (fk) {
        if ((e = cudaEventRecord(fk->fork_ev, st)) != cudaSuccess) return cuda_fail(e, "fork");
        for (int i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(fk->s[i], fk->fork_ev, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    }
    qai_status s = QAI_OK;
    {
        LaunchSink sink(kernels);
        for (size_t k = 0; k < order.size() && s == QAI_OK; ++k) {
            const Field& f = bt.f[order[k]];
            s = run_plain(f.q, f.out, f.sh, f.m, ws + f.ws_off, f.lay, fk ? fk->s[k % ns] : st);
        }
    }
    if (fk) {  // join, also after an error, so no stream is left forked
        for (int i = 0; i < ns; ++i) {
            if ((e = cudaEventRecord(fk->join_ev[i], fk->s[i])) != cudaSuccess && s == QAI_OK) s = cuda_fail(e, "join");
            if ((e = cudaStreamWaitEvent(st, fk->join_ev[i], 0)) != cudaSuccess && s == QAI_OK) s = cuda_fail(e, "join");
        }
    }
    return s;
}

// ---- the grouped persistent form (rank 2 and 3) ----------------------------

struct Tune {
    int order = 1;       // 1: largest field first, 0: as given
    int gran_log2 = 16;  // points per work item of the grid-stride kernels: 2^gran_log2
    int col_rpb = 0;     // column tiles: rows per band (0: the plain call's tiles)
    int col_w = 16;      // column tiles: the largest width
};

enum Kind { kKDetect, kKNear, kKExpand, kKPackS, kKRoute, kKRow, kKCol };

// One grouped launch: its kernel, its fields' virtual blocks, gates and
// argument structs (arg_size bytes each).
struct GLaunch {
    int kind = 0, mode = 0, phase = 0, in_bytes = 0, fin = 0, narrow = 0, W = 0, B = 0, warps = 0, max_nx = 0;
    size_t smem = 0, arg_size = 0;
    std::vector<int> vb;
    std::vector<const int*> gate;
    std::vector<unsigned char> args;
    size_t table_off = 0;  // of the argument structs, from the header's start
    bool same(const GLaunch& o) const
    {
        return kind == o.kind && mode == o.mode && phase == o.phase && in_bytes == o.in_bytes && fin == o.fin &&
               narrow == o.narrow && W == o.W && B == o.B && warps == o.warps;
    }
};

struct GPlan {
    std::vector<GLaunch> launches;
    size_t cursors_off = 0, ctr_off = 0, tables_off = 0, zero_bytes = 0, table_bytes = 0;
    std::vector<unsigned char> tables;  // host image of the tables
};

int sm_count()
{
    int dev = 0, n = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// The grouped launches of the rank-2 and rank-3 fields, in the plain
// sequence's order; `ws` is the device workspace (the header at its start).
qai_status plan_grouped(const Batch& bt, const Tune& tn, char* ws, GPlan& gp)
{
    gp = GPlan{};
    std::vector<int> order;
    for (int r = 2; r <= 3; ++r) order.insert(order.end(), bt.group[r].begin(), bt.group[r].end());
    if (order.empty()) return QAI_OK;
    if (tn.order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bt.f[a].sh.N > bt.f[b].sh.N; });
    const int nf = (int)bt.f.size();
    gp.cursors_off = 0;
    gp.ctr_off = align256((size_t)(kLaunchesPerField * nf + 64) * 4);
    gp.tables_off = gp.ctr_off + align256((size_t)nf * kCtrWords * 4);
    gp.zero_bytes = gp.tables_off;
    const int sms = sm_count();
    const int64_t gran = 1LL << tn.gran_log2;
    auto clampv = [](int64_t v, int64_t hi) { return (int)std::max<int64_t>(1, std::min<int64_t>(v, hi)); };

    std::vector<PlainArgs> pa(order.size());
    for (size_t j = 0; j < order.size(); ++j) {
        const Field& f = bt.f[order[j]];
        int* ctr = reinterpret_cast<int*>(ws + gp.ctr_off) + (size_t)j * kCtrWords;
        if (!plain_args(f.q, f.out, f.sh, f.m, ws + f.ws_off, f.lay, ctr, &pa[j]))
            return fail(QAI_ERR_SHAPE, "field %d: line length does not fit shared memory", f.index);
    }
    // a stage: one launch per distinct key, at most kGroupMax fields each
    std::vector<GLaunch> stage;
    auto add = [&](const GLaunch& key, int vb, const int* gate, const void* arg, size_t size) {
        GLaunch* g = nullptr;
        for (GLaunch& c : stage)
            if (c.same(key) && (int)c.vb.size() < kGroupMax) g = &c;
        if (!g) {
            stage.push_back(key);
            g = &stage.back();
            g->arg_size = size;
        }
        g->vb.push_back(vb);
        g->gate.push_back(gate);
        const unsigned char* b = static_cast<const unsigned char*>(arg);
        g->args.insert(g->args.end(), b, b + size);
        g->smem = std::max(g->smem, key.smem);
        g->max_nx = std::max(g->max_nx, key.max_nx);
    };
    auto flush = [&]() {
        for (GLaunch& g : stage) gp.launches.push_back(std::move(g));
        stage.clear();
    };
    auto for_fields = [&](auto&& fn) {
        for (size_t j = 0; j < order.size(); ++j) fn(bt.f[order[j]], pa[j]);
        flush();
    };
    auto K = [](int kind) { GLaunch g; g.kind = kind; return g; };
    auto items = [&](const Field& f, int64_t cap) { return clampv(((int64_t)f.sh.N + gran - 1) / gran, cap); };
    auto ctr_of = [](const PlainArgs& p, int w) -> const int* { return p.la.ctr + w; };

    // step A (the fast pass; with sign rule FIRST the exact one alone)
    const bool fast = bt.f[order[0]].m.sign_rule == 0;
    for_fields([&](const Field& f, const PlainArgs& p) {
        GLaunch k = K(kKDetect); k.mode = fast ? 0 : 1;
        add(k, items(f, 8 * sms), nullptr, &p.la, sizeof p.la);
    });
    if (fast) for_fields([&](const Field& f, const PlainArgs& p) {
        GLaunch k = K(kKDetect); k.mode = 2;
        add(k, items(f, 8 * sms), ctr_of(p, kCtrWide), &p.la, sizeof p.la);
    });
    for_fields([&](const Field& f, const PlainArgs& p) {
        add(K(kKNear), items(f, 8 * sms), nullptr, &p.la, sizeof p.la);
    });
    // the separable first EDT, where the bounded search fell short; every row
    // launch takes the warps the widest field allows
    int max_nx = 0;
    for (int j : order) max_nx = std::max(max_nx, bt.f[j].sh.nx);
    const int warps = rowpass_warps(max_nx);
    auto row = [&](int phase, const Field& f, const RowArgs& r, const int* gate) {
        GLaunch k = K(kKRow); k.phase = phase; k.warps = warps; k.max_nx = max_nx;
        const int64_t rows = (int64_t)f.sh.nz * f.sh.ny;
        add(k, clampv((rows + warps - 1) / warps, 4 * sms), gate, &r, sizeof r);
    };
    // a column stage: the fields with the same pass instance share one tile
    // shape -- bands from the longest line (no more than the shortest one has
    // rows), the widest tile up to the tuned width that fits
    struct ColItem { const Field* f; ColArgs c; int in_bytes; bool fin; const int* gate; };
    auto col_stage = [&](std::vector<ColItem>& its, int phase) -> qai_status {
        const int rpb = tn.col_rpb > 0 ? tn.col_rpb : 32;
        std::vector<int> done(its.size(), 0);
        for (size_t i = 0; i < its.size(); ++i) {
            if (done[i]) continue;
            const ColItem& it = its[i];
            const int wmax = tn.col_rpb > 0 ? tn.col_w : (it.in_bytes == 4 ? 32 : 8);  // the plain call's widths
            int maxL = 0, minL = 1 << 30;
            std::vector<size_t> same;
            for (size_t j = i; j < its.size(); ++j) {
                const ColItem& o = its[j];
                if (done[j] || o.in_bytes != it.in_bytes || o.fin != it.fin || o.c.narrow != it.c.narrow) continue;
                same.push_back(j);
                maxL = std::max(maxL, o.c.L);
                minL = std::min(minL, o.c.L);
            }
            ColConfig cfg{};
            cfg.B = std::max(2, std::min(std::min(32, minL), (maxL + rpb - 1) / rpb));
            for (int W = wmax; W >= 4; W >>= 1) {
                if (W * cfg.B > 512) continue;
                const size_t sm = (size_t)maxL * W * (it.in_bytes + 2) + (size_t)4 * cfg.B * W * 2 + (size_t)W * 2;
                if (sm <= 200 * 1024) { cfg.W = W; cfg.smem = (sm + 15) & ~(size_t)15; break; }
            }
            if (!cfg.W) return fail(QAI_ERR_SHAPE, "column tiles do not fit shared memory");
            for (size_t j : same) {
                done[j] = 1;
                ColItem& o = its[j];
                const int64_t gx = (int64_t)(o.f->sh.nx - 1) * (o.f->sh.nx - 1);
                const int64_t gxy = gx + (int64_t)(o.f->sh.ny - 1) * (o.f->sh.ny - 1);
                const int narrow = o.c.narrow;
                prepare_colpass(o.c, o.in_bytes, cfg, o.in_bytes == 2 ? gx : gxy);
                if (o.c.narrow != narrow) return fail(QAI_ERR_INTERNAL, "column pass arithmetic changed");
                GLaunch k = K(kKCol); k.phase = phase; k.fin = o.fin; k.in_bytes = o.in_bytes; k.narrow = narrow;
                k.W = cfg.W; k.B = cfg.B; k.smem = cfg.smem;
                const int64_t tiles = (int64_t)((o.c.C + cfg.W - 1) / cfg.W) * o.c.P;
                add(k, clampv(tiles, 4 * sms), o.gate, &o.c, sizeof o.c);
            }
        }
        flush();
        return QAI_OK;
    };
    auto col_phase = [&](int phase) -> qai_status {
        std::vector<ColItem> it1, it2;
        for (size_t j = 0; j < order.size(); ++j) {
            const Field& f = bt.f[order[j]];
            const PlainArgs& p = pa[j];
            const int* gate = ctr_of(p, phase == 1 ? kCtrLocalFail : kCtrDense);
            it1.push_back({&f, phase == 1 ? p.c1[0] : p.c2[0], 2, f.sh.rank == 2, gate});
            if (f.sh.rank == 3) it2.push_back({&f, phase == 1 ? p.c1[1] : p.c2[1], 4, true, gate});
        }
        qai_status st = col_stage(it1, phase);
        return st == QAI_OK ? col_stage(it2, phase) : st;
    };
    for_fields([&](const Field& f, const PlainArgs& p) { row(1, f, p.r1, ctr_of(p, kCtrLocalFail)); });
    qai_status st = col_phase(1);
    if (st != QAI_OK) return st;
    for_fields([&](const Field& f, const PlainArgs& p) {
        GLaunch k = K(kKPackS); k.mode = 1;
        add(k, items(f, 4 * sms), ctr_of(p, kCtrLocalFail), &p.la, sizeof p.la);
    });
    // the signed-point route (vb > 0: the plain call's grid, which some of
    // these kernels' decisions depend on)
    auto route = [&](RouteKernel rk, int64_t vb, int gate_word) {
        for_fields([&](const Field& f, const PlainArgs& p) {
            GLaunch k = K(kKRoute); k.mode = (int)rk;
            add(k, vb > 0 ? (int)vb : items(f, 2 * sms), ctr_of(p, gate_word), &p.ra, sizeof p.ra);
        });
    };
    route(kRouteB2Sparse, 0, kCtrQueries);
    route(kRouteBruteSparse, 2 * sms, kCtrQueries);
    route(kRouteB2Map, 0, kCtrBitmap);
    route(kRouteQuery, 4 * sms, kCtrBitmap);
    route(kRouteQueryMid, 4 * sms, kCtrBitmap);
    route(kRouteB2List, 2 * sms, kCtrBitmap);
    route(kRouteBrute, 2 * sms, kCtrBitmap);
    for_fields([&](const Field& f, const PlainArgs& p) {
        GLaunch k = K(kKExpand); k.mode = 1;
        add(k, items(f, 4 * sms), ctr_of(p, kCtrDense), &p.la, sizeof p.la);
    });
    // the dense second EDT, where the route handed the field over
    for_fields([&](const Field& f, const PlainArgs& p) { row(2, f, p.r2, ctr_of(p, kCtrDense)); });
    if ((st = col_phase(2)) != QAI_OK) return st;

    if (gp.launches.size() > (size_t)(kLaunchesPerField * nf + 64)) return fail(QAI_ERR_INTERNAL, "too many launches");
    size_t off = 0;
    for (GLaunch& g : gp.launches) {
        g.table_off = gp.tables_off + off;
        off = (off + g.args.size() + 15) & ~(size_t)15;
    }
    gp.table_bytes = off;
    if (gp.tables_off + off > bt.header) return fail(QAI_ERR_INTERNAL, "argument tables exceed the header");
    gp.tables.assign(off, 0);
    for (const GLaunch& g : gp.launches)
        std::memcpy(gp.tables.data() + (g.table_off - gp.tables_off), g.args.data(), g.args.size());
    return QAI_OK;
}

const char* group_name(const GLaunch& g)
{
    static const char* route[] = {"group_b2sparse", "group_brute_sparse", "group_b2map", "group_query",
                                  "group_query_mid", "group_b2list", "group_brute"};
    switch (g.kind) {
    case kKDetect: return g.mode == 2 ? "group_detect_exact" : "group_detect";
    case kKNear: return "group_near";
    case kKExpand: return "group_expand";
    case kKPackS: return "group_pack_s";
    case kKRoute: return route[g.mode];
    case kKRow: return g.phase == 1 ? "group_rowpass1" : "group_rowpass2";
    default: return g.phase == 1 ? "group_colpass1" : "group_colpass2";
    }
}

// The grouped launches on `st` (the tables already in place): the cursors
// and counters cleared, then one kernel per launch (counted and, while
// profiling, timed by name).
qai_status launch_grouped(const GPlan& gp, char* ws, cudaStream_t st)
{
    if (gp.launches.empty()) return QAI_OK;
    cudaError_t e = cudaMemsetAsync(ws, 0, gp.zero_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "clear cursors");
    int* cursors = reinterpret_cast<int*>(ws + gp.cursors_off);
    for (size_t i = 0; i < gp.launches.size(); ++i) {
        const GLaunch& g = gp.launches[i];
        GroupQueue q{};
        q.n = (int)g.vb.size();
        q.cursor = cursors + i;
        q.args = ws + g.table_off;
        for (int f = 0; f < q.n; ++f) {
            q.vb[f] = g.vb[f];
            q.gate[f] = g.gate[f];
        }
        e = timed_call(group_name(g), 0.0, st, [&]() -> cudaError_t {
            switch (g.kind) {
            case kKDetect: return launch_group_detect(q, g.mode, st);
            case kKNear: return launch_group_near(q, st);
            case kKExpand: return launch_group_expand(q, g.mode, st);
            case kKPackS: return launch_group_pack_s(q, g.mode, st);
            case kKRoute: return launch_group_route((RouteKernel)g.mode, q, st);
            case kKRow: return launch_group_rowpass(q, g.phase, g.warps, g.max_nx, st);
            default:
                return launch_group_colpass(q, g.phase, g.in_bytes, g.fin != 0, g.narrow != 0, g.W, g.B, g.smem, st);
            }
        });
        if (e != cudaSuccess) return cuda_fail(e, "grouped launch");
    }
    return QAI_OK;
}

std::unordered_map<uint64_t, Tune> g_tuned_grouped;  // rank-2/3 shape signature -> tuning

uint64_t grouped_signature(const Batch& bt)
{
    return group_signature(bt, 2) ^ (group_signature(bt, 3) * 1099511628211ull);
}

Tune tuned_grouped(uint64_t sig)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned_grouped.find(sig);
    return it == g_tuned_grouped.end() ? Tune() : it->second;
}

// Every group's launches on `st`: rank 2 and 3 as the grouped launches of
// `gp` (its tables already in place) when given, else per field.
qai_status launch_all(const Batch& bt, const GroupCfg cfgs[4], char* ws, cudaStream_t st, int* kernels,
                      const GPlan* gp)
{
    if (gp) {
        qai_status s;
        {
            LaunchSink sink(kernels);
            s = launch_grouped(*gp, ws, st);
        }
        if (s != QAI_OK) return s;
        return launch_group(bt, 1, cfgs[1], ws, st, kernels);
    }
    for (int rank = 3; rank >= 1; --rank) {
        qai_status s = launch_group(bt, rank, cfgs[rank], ws, st, kernels);
        if (s != QAI_OK) return s;
    }
    return QAI_OK;
}

qai_status check_ws(const Batch& bt, void* d_ws, size_t ws_bytes)
{
    if (!d_ws) return fail(QAI_ERR_INVALID_ARG, "d_ws must be non-NULL");
    if (ws_bytes < bt.ws_total)
        return fail(QAI_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, bt.ws_total);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return QAI_OK;
}

}  // namespace

extern "C" {

qai_status qai_workspace_size_batched(int n, const int32_t* ranks, const int64_t* dims, size_t* bytes)
{
    if (!bytes || !ranks || !dims || n < 1) return fail(QAI_ERR_INVALID_ARG, "bad arguments");
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        Shape sh;
        qai_status s = make_shape(ranks[i], dims + 3 * i, &sh);
        if (s != QAI_OK) return s;
        off = align256(off + layout_for(sh, 0).total);
    }
    *bytes = off + header_bytes(n);
    return QAI_OK;
}

qai_status qai_mitigate_batched(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                                const int64_t* dims, const double* eb, const qai_params* params, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream)
{
    qai::set_last_error("");
    Batch bt;
    qai_status s = plan(n, d_q, d_out, ranks, dims, eb, params, bt);
    if (s != QAI_OK) return s;
    if ((s = check_ws(bt, d_ws, ws_bytes)) != QAI_OK) return s;
    GroupCfg cfgs[4];
    for (int r = 1; r <= 3; ++r) cfgs[r] = tuned_cfg(group_signature(bt, r));
    char* ws = static_cast<char*>(d_ws);

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return cuda_fail(cudaGetLastError(), "stream query");
    int kernels = 0;
    if (cs != cudaStreamCaptureStatusNone) {  // the caller captures: record per-field sequences into its graph
        s = launch_all(bt, cfgs, ws, stream, &kernels, nullptr);
        for (int k = 0; k < kernels; ++k) count_launch();
        return s;
    }
    const Tune tn = tuned_grouped(grouped_signature(bt));
    // key of the cached graph: every argument that reaches a kernel
    uint64_t key = fnv(&n, sizeof n, 1469598103934665603ull);
    key = fnv(d_q, n * sizeof(void*), key);
    key = fnv(d_out, n * sizeof(void*), key);
    key = fnv(ranks, n * sizeof(int32_t), key);
    key = fnv(dims, 3 * n * sizeof(int64_t), key);
    key = fnv(eb, n * sizeof(double), key);
    qai_params pv;
    if (params) pv = *params; else qai_default_params(&pv);
    key = fnv(&pv, sizeof pv, key);
    key = fnv(&d_ws, sizeof d_ws, key);
    key = fnv(cfgs, sizeof cfgs, key);
    key = fnv(&tn, sizeof tn, key);
    key = fnv(&stream, sizeof stream, key);

    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (size_t i = 0; i < g_graphs.size(); ++i) {
            if (g_graphs[i].key == key) {
                GraphEntry e = g_graphs[i];
                g_graphs.erase(g_graphs.begin() + i);
                g_graphs.push_back(e);
                exec = e.exec;
                kernels = e.kernels;
                break;
            }
        }
    }
    if (!exec) {
        GPlan gp;
        void* host_tables = nullptr;
        if (bt.grouped) {
            if ((s = plan_grouped(bt, tn, ws, gp)) != QAI_OK) return s;
            if (gp.table_bytes) {
                cudaError_t eh = cudaMallocHost(&host_tables, gp.table_bytes);
                if (eh != cudaSuccess) return cuda_fail(eh, "pinned argument tables");
                std::memcpy(host_tables, gp.tables.data(), gp.table_bytes);
            }
        }
        // Capture on a private stream (the caller's may be the legacy default
        // stream, which cannot capture); the graph is launched on `stream`.
        thread_local cudaStream_t cap = nullptr;
        if (!cap) {
            cudaError_t ec = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (ec != cudaSuccess) { cap = nullptr; cudaFreeHost(host_tables); return cuda_fail(ec, "capture stream"); }
        }
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaFreeHost(host_tables); return cuda_fail(e, "begin capture"); }
        if (host_tables) {
            e = cudaMemcpyAsync(ws + gp.tables_off, host_tables, gp.table_bytes, cudaMemcpyHostToDevice, cap);
            if (e != cudaSuccess) s = cuda_fail(e, "argument tables");
        }
        if (s == QAI_OK) s = launch_all(bt, cfgs, ws, cap, &kernels, bt.grouped ? &gp : nullptr);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (s != QAI_OK || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaFreeHost(host_tables);
            return s != QAI_OK ? s : cuda_fail(e2, "end capture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { cudaFreeHost(host_tables); return cuda_fail(e, "graph instantiate"); }
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_graphs.size() >= kMaxGraphs) {
            cudaGraphExecDestroy(g_graphs.front().exec);
            cudaFreeHost(g_graphs.front().host_tables);
            g_graphs.erase(g_graphs.begin());
        }
        g_graphs.push_back({key, exec, kernels, host_tables});
    }
    cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    for (int k = 0; k < kernels; ++k) count_launch();
    return QAI_OK;
}

qai_status qai_autotune_batched(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                                const int64_t* dims, const double* eb, const qai_params* params, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream, qai_batch_choice* choices)
{
    qai::set_last_error("");
    Batch bt;
    qai_status s = plan(n, d_q, d_out, ranks, dims, eb, params, bt);
    if (s != QAI_OK) return s;
    if ((s = check_ws(bt, d_ws, ws_bytes)) != QAI_OK) return s;
    char* ws = static_cast<char*>(d_ws);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "event create");
    if (choices) std::memset(choices, 0, 3 * sizeof(qai_batch_choice));
    // time `run` (one warm-up, then three runs): milliseconds per run
    auto timed_runs = [&](auto&& run, float* ms) -> qai_status {
        qai_status st = run();
        if (st != QAI_OK) return st;
        cudaEventRecord(e0, stream);
        for (int rep = 0; rep < 3 && st == QAI_OK; ++rep) st = run();
        cudaEventRecord(e1, stream);
        if (st != QAI_OK) return st;
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune sync");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= 3.f;
        return QAI_OK;
    };
    static const GroupCfg cands[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {0, 1}, {0, 2}, {0, 4}, {0, 8}};
    for (int rank = 1; rank <= 3 && s == QAI_OK; ++rank) {
        if (bt.group[rank].empty() || (rank > 1 && bt.grouped)) continue;
        float best_ms = 1e30f;
        GroupCfg best;
        for (const GroupCfg& c : cands) {
            if (rank == 1 && c.streams != 1) continue;  // rank 1: one grouped launch per phase
            float ms = 0.f;
            int kernels = 0;
            s = timed_runs([&] { return launch_group(bt, rank, c, ws, stream, &kernels); }, &ms);
            if (s != QAI_OK) break;
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        if (s != QAI_OK) break;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            g_tuned[group_signature(bt, rank)] = best;
        }
        if (choices) {
            qai_batch_choice& ch = choices[rank - 1];
            ch.rank = rank;
            ch.fields = (int32_t)bt.group[rank].size();
            ch.streams = best.streams;
            ch.order = best.order;
            ch.ms = best_ms;
        }
    }
    if (s == QAI_OK && bt.grouped && (!bt.group[2].empty() || !bt.group[3].empty())) {
        // greedy: the queue order, then the work-item size, then the column tiles
        Tune best;
        float best_ms = 1e30f;
        int best_launches = 0;
        auto trial = [&](const Tune& t) -> qai_status {
            GPlan gp;
            qai_status st = plan_grouped(bt, t, ws, gp);
            if (st != QAI_OK) return st == QAI_ERR_SHAPE ? QAI_OK : st;  // tiles that do not fit: skipped
            cudaError_t e = cudaMemcpyAsync(ws + gp.tables_off, gp.tables.data(), gp.table_bytes,
                                            cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_fail(e, "argument tables");
            float ms = 0.f;
            st = timed_runs([&] { return launch_grouped(gp, ws, stream); }, &ms);
            if (st != QAI_OK) return st;
            if (ms < best_ms) { best_ms = ms; best = t; best_launches = (int)gp.launches.size(); }
            return QAI_OK;
        };
        Tune t;
        for (int o : {1, 0}) {
            if (s != QAI_OK) break;
            t.order = o;
            s = trial(t);
        }
        t = best;
        for (int g : {14, 15, 17, 18}) {
            if (s != QAI_OK) break;
            t.gran_log2 = g;
            s = trial(t);
        }
        t = best;
        static const int tiles[][2] = {{32, 8}, {32, 16}, {32, 32}, {16, 8}, {16, 16}, {64, 16}, {64, 32}};
        for (const auto& c : tiles) {
            if (s != QAI_OK) break;
            t.col_rpb = c[0];
            t.col_w = c[1];
            s = trial(t);
        }
        if (s == QAI_OK) {
            {
                std::lock_guard<std::mutex> lk(g_mu);
                g_tuned_grouped[grouped_signature(bt)] = best;
            }
            if (choices) {
                for (int rank = 2; rank <= 3; ++rank) {
                    qai_batch_choice& ch = choices[rank - 1];
                    ch.rank = rank;
                    ch.fields = (int32_t)bt.group[rank].size();
                    ch.streams = 0;
                    ch.order = best.order;
                    ch.ms = best_ms;
                    ch.grouped = 1;
                    ch.tile_w = best.col_rpb ? best.col_w : 0;
                    ch.rows_per_band = best.col_rpb;
                    ch.points_per_block = 1 << best.gran_log2;
                    ch.launches = best_launches;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

}  // extern "C"
